"""qslab: long-range electrostatics of quasi-2D slabs on one GB300 GPU.

Python binding of the C ABI in include/qslab.h (argument marshalling only:
every step of the computation runs in the CUDA library libqslab.so). The
module-level functions carry the C names; ``QSlab`` wraps a context for
torch tensors, and ``SlabEnergy`` is the autograd function whose backward is
the exact adjoint of the long-range energy (dE/dr = -F, dE/dq = phi; E is a
quadratic form in q).

Method: Gan, Gao, Liang, Xu, "Fast algorithm for quasi-2D Coulomb systems"
(arXiv 2403.01521): the SOE-Ewald2D long-range part with the full k-sum
(Algorithm 1) or the random-batch importance sampler (Algorithm 2).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build
from .soe import load_soe  # noqa: F401  (tables are method parameters)

QSLAB_FP64 = 0
QSLAB_FP32C = 1
QSLAB_SAMPLER_IID = 0
QSLAB_SAMPLER_METROPOLIS = 1
# status codes (include/qslab.h)
QSLAB_OK = 0
QSLAB_ERR_INVALID_ARG = -1
QSLAB_ERR_NOT_CONFIGURED = -2
QSLAB_ERR_NONFINITE = -3
QSLAB_ERR_Z_OUT_OF_RANGE = -4
QSLAB_ERR_NONNEUTRAL = -5
QSLAB_ERR_ALLOC = -6
QSLAB_ERR_CUDA = -7
QSLAB_ERR_TIMEOUT = -8
QSLAB_ERR_TOO_LARGE = -9
QSLAB_ERR_INTERNAL = -10
_PREC = {"fp64": QSLAB_FP64, "fp32c": QSLAB_FP32C}

_lib = None


class QslabError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib.qslab_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} (code {code})")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libqslab.so (building it first if allowed). Raises if the CUDA
    library cannot be built or loaded: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    # QSLAB_LIBRARY=debug selects the debug build (internal index checks)
    debug = os.environ.get("QSLAB_LIBRARY", "") == "debug"
    path = _build.DEBUG_LIB if debug else _build.LIB
    if not _build.up_to_date(path):
        if not build_if_missing:
            raise RuntimeError(f"{os.path.basename(path)} missing or stale at {path}")
        _build.build(debug=debug)
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.c_double
    I = ctypes.c_int
    sig = {
        "qslab_create": ([ctypes.POINTER(P), I, I], I),
        "qslab_destroy": ([P], None),
        "qslab_set_box": ([P, D, D, D], I),
        "qslab_set_alpha": ([P, D], I),
        "qslab_set_kcut": ([P, D], I),
        "qslab_set_rbe": ([P, I, ctypes.c_uint64], I),
        "qslab_set_soe": ([P, I, P, P, P, P], I),
        "qslab_set_neutrality_tol": ([P, D], I),
        "qslab_set_tuning": ([P, I, I], I),
        "qslab_compute": ([P, ctypes.c_int64, P, P, P, P, P, P], I),
        "qslab_compute_host": ([P, ctypes.c_int64, P, P, P, P, P, P], I),
        "qslab_compute_static": ([P, ctypes.c_int64, P, P, P, P, P, P], I),
        "qslab_compute_batched": ([P, I, P, P, P, P, P, P, P, P], I),
        "qslab_compute_virial": ([P, ctypes.c_int64, P, P, P, P, P, P, P], I),
        "qslab_compute_energy": ([P, ctypes.c_int64, P, P, P, P], I),
        "qslab_compute_batched_energy": ([P, I, P, P, P, P, P, P], I),
        "qslab_compute_adjoint": ([P, P, P, P], I),
        "qslab_measure_peaks": ([I, P, P], I),
        "qslab_compute_batched_virial": ([P, I, P, P, P, P, P, P, P, P, P], I),
        "qslab_compute_realspace_virial": ([P, ctypes.c_int64, P, P, P, P, P, P, P], I),
        "qslab_autotune": ([P, I, P, P, P, P, P, I, P, P], I),
        "qslab_set_rcut": ([P, D], I),
        "qslab_set_walls": ([P, D, D, I, P, P, P], I),
        "qslab_set_rbe_sampler": ([P, I, I], I),
        "qslab_md_configure": ([P, D, D, D, D, D, D, D, D, ctypes.c_uint64], I),
        "qslab_md_forces": ([P, ctypes.c_int64, P, P, P, P, P, P], I),
        "qslab_md_step": ([P, ctypes.c_int64, P, P, P, P, I, P, P], I),
        "qslab_md_set_step": ([P, ctypes.c_uint64], I),
        "qslab_md_get_step": ([P, P], I),
        "qslab_clear_walls": ([P], I),
        "qslab_compute_realspace": ([P, ctypes.c_int64, P, P, P, P, P, P], I),
        "qslab_get_sampled_modes": ([P, P, P], I),
        "qslab_get_rng_state": ([P, P, P], I),
        "qslab_set_rng_state": ([P, ctypes.c_uint64, ctypes.c_uint64], I),
        "qslab_num_modes": ([P], I),
        "qslab_last_status": ([P], I),
        "qslab_set_timing": ([P, I], I),
        "qslab_get_timings": ([P, P, P], I),
        "qslab_strerror": ([I], ctypes.c_char_p),
        "qslab_debug_alloc_count": ([], ctypes.c_longlong),
        "qslab_debug_fail_alloc": ([I], I),
        "qslab_debug_stall_sort": ([I], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(rc: int, where: str):
    if rc != 0:
        raise QslabError(rc, where)


# ---------------------------------------------------------------- C names


def qslab_create(device: int = 0, prec: int = QSLAB_FP64) -> int:
    lib = load()
    h = ctypes.c_void_p()
    _check(lib.qslab_create(ctypes.byref(h), device, prec), "qslab_create")
    return h.value


def qslab_destroy(h: int):
    load().qslab_destroy(h)


def qslab_set_box(h, Lx, Ly, Lz):
    _check(load().qslab_set_box(h, Lx, Ly, Lz), "qslab_set_box")


def qslab_set_alpha(h, alpha):
    _check(load().qslab_set_alpha(h, alpha), "qslab_set_alpha")


def qslab_set_kcut(h, kc):
    _check(load().qslab_set_kcut(h, kc), "qslab_set_kcut")


def qslab_set_rbe(h, P, seed):
    _check(load().qslab_set_rbe(h, int(P), int(seed)), "qslab_set_rbe")


def qslab_set_soe(h, s, w):
    s = np.asarray(s, complex)
    w = np.asarray(w, complex)
    arrs = [np.ascontiguousarray(a, np.float64) for a in (s.real, s.imag, w.real, w.imag)]
    ptrs = [a.ctypes.data for a in arrs]
    _check(load().qslab_set_soe(h, len(s), *ptrs), "qslab_set_soe")


def qslab_set_neutrality_tol(h, tol):
    _check(load().qslab_set_neutrality_tol(h, tol), "qslab_set_neutrality_tol")


def qslab_set_tuning(h, chunk=0, modes_per_cta=0):
    _check(load().qslab_set_tuning(h, chunk, modes_per_cta), "qslab_set_tuning")


def qslab_compute(h, N, pos_ptr, q_ptr, energy_ptr, phi_ptr, force_ptr, stream_ptr):
    _check(load().qslab_compute(h, N, pos_ptr, q_ptr, energy_ptr, phi_ptr, force_ptr,
                                stream_ptr), "qslab_compute")


def qslab_compute_host(h, N, pos_ptr, q_ptr, energy_ptr, phi_ptr, force_ptr, stream_ptr):
    _check(load().qslab_compute_host(h, N, pos_ptr, q_ptr, energy_ptr, phi_ptr, force_ptr,
                                     stream_ptr), "qslab_compute_host")


def qslab_compute_static(h, N, pos_ptr, q_ptr, energy_ptr, phi_ptr, force_ptr, stream_ptr):
    """qslab_compute() for callers that cannot allocate device memory: all
    scratch comes from the library's fixed 64 MiB device array. Waits for the
    stream and raises on any error, including device-side input errors."""
    _check(load().qslab_compute_static(h, N, pos_ptr, q_ptr, energy_ptr, phi_ptr, force_ptr,
                                       stream_ptr), "qslab_compute_static")


def qslab_compute_batched(h, offsets, boxes, pos_ptr, q_ptr, energies_ptr, phi_ptr, force_ptr,
                          stream_ptr):
    """R slabs in one call. offsets: R+1 int64 (host), boxes: R x 3 float64
    (host); the other arguments as for qslab_compute()."""
    off = np.ascontiguousarray(offsets, np.int64)
    box = np.ascontiguousarray(boxes, np.float64).reshape(-1, 3)
    R = off.shape[0] - 1
    if box.shape[0] != R:
        raise ValueError("boxes must have one row per replica")
    _check(load().qslab_compute_batched(h, R, off.ctypes.data, box.ctypes.data, pos_ptr, q_ptr,
                                        energies_ptr, phi_ptr, force_ptr, stream_ptr),
           "qslab_compute_batched")


def qslab_compute_virial(h, N, pos_ptr, q_ptr, energy_ptr, phi_ptr, force_ptr, virial_ptr,
                         stream_ptr):
    _check(load().qslab_compute_virial(h, N, pos_ptr, q_ptr, energy_ptr, phi_ptr, force_ptr,
                                       virial_ptr, stream_ptr), "qslab_compute_virial")


def qslab_measure_peaks(device=0, stream_ptr=None):
    """Measured lane-operation rates of the device (ops/s): FP32 FMA, packed
    FP32 FMA (two per instruction), FP64 FMA, ex2.approx."""
    out = np.zeros(4)
    _check(load().qslab_measure_peaks(int(device), out.ctypes.data, stream_ptr),
           "qslab_measure_peaks")
    return {"fp32_fma": float(out[0]), "fp32_ffma2": float(out[1]), "fp64_fma": float(out[2]),
            "ex2": float(out[3])}


def qslab_compute_energy(h, N, pos_ptr, q_ptr, energy_ptr, stream_ptr):
    """Energy only (forward sums); leaves the workspace for qslab_compute_adjoint."""
    _check(load().qslab_compute_energy(h, N, pos_ptr, q_ptr, energy_ptr, stream_ptr),
           "qslab_compute_energy")


def qslab_compute_batched_energy(h, offsets, boxes, pos_ptr, q_ptr, energies_ptr, stream_ptr):
    off = np.ascontiguousarray(offsets, np.int64)
    box = np.ascontiguousarray(boxes, np.float64).reshape(-1, 3)
    R = off.shape[0] - 1
    if box.shape[0] != R:
        raise ValueError("boxes must have one row per replica")
    _check(load().qslab_compute_batched_energy(h, R, off.ctypes.data, box.ctypes.data, pos_ptr,
                                               q_ptr, energies_ptr, stream_ptr),
           "qslab_compute_batched_energy")


def qslab_compute_adjoint(h, phi_ptr, force_ptr, stream_ptr):
    """phi = dE/dq and F = -dE/dr of the last energy-only call."""
    _check(load().qslab_compute_adjoint(h, phi_ptr, force_ptr, stream_ptr),
           "qslab_compute_adjoint")


def qslab_compute_batched_virial(h, offsets, boxes, pos_ptr, q_ptr, energies_ptr, phi_ptr,
                                 force_ptr, virial_ptr, stream_ptr):
    off = np.ascontiguousarray(offsets, np.int64)
    box = np.ascontiguousarray(boxes, np.float64).reshape(-1, 3)
    R = off.shape[0] - 1
    if box.shape[0] != R:
        raise ValueError("boxes must have one row per replica")
    _check(load().qslab_compute_batched_virial(h, R, off.ctypes.data, box.ctypes.data, pos_ptr,
                                               q_ptr, energies_ptr, phi_ptr, force_ptr,
                                               virial_ptr, stream_ptr),
           "qslab_compute_batched_virial")


def qslab_compute_realspace_virial(h, N, pos_ptr, q_ptr, energy_ptr, phi_ptr, force_ptr,
                                   virial_ptr, stream_ptr):
    _check(load().qslab_compute_realspace_virial(h, N, pos_ptr, q_ptr, energy_ptr, phi_ptr,
                                                 force_ptr, virial_ptr, stream_ptr),
           "qslab_compute_realspace_virial")


def qslab_autotune(h, offsets, boxes, pos_ptr, q_ptr, stream_ptr, reps=3):
    """Time the candidate launch shapes on these inputs and keep the fastest;
    returns (chunk, modes_per_cta)."""
    off = np.ascontiguousarray(offsets, np.int64)
    box = np.ascontiguousarray(boxes, np.float64).reshape(-1, 3)
    R = off.shape[0] - 1
    if box.shape[0] != R:
        raise ValueError("boxes must have one row per replica")
    L = ctypes.c_int()
    kr = ctypes.c_int()
    _check(load().qslab_autotune(h, R, off.ctypes.data, box.ctypes.data, pos_ptr, q_ptr,
                                 stream_ptr, int(reps), ctypes.addressof(L), ctypes.addressof(kr)),
           "qslab_autotune")
    return L.value, kr.value


def qslab_set_rcut(h, rc):
    _check(load().qslab_set_rcut(h, float(rc)), "qslab_set_rcut")


def qslab_set_walls(h, sigma_bot, sigma_top, modes=None, bot=None, top=None):
    """Charged walls (Section 2.4, Thm 2.4): uniform densities sigma_bot at
    z = 0 and sigma_top at z = Lz, plus Fourier modes: modes = [(mx, my), ...]
    (each pair (m, -m) once), bot/top = complex coefficients c_w of
    sigma(rho) = sigma0 + sum_w 2 Re[c_w e^{i k_w.rho}]."""
    modes = np.ascontiguousarray(np.zeros((0, 2)) if modes is None else modes, dtype=np.int32).reshape(-1, 2)
    nw = modes.shape[0]
    b = np.asarray([] if bot is None else bot, dtype=complex).reshape(-1)
    t = np.asarray([] if top is None else top, dtype=complex).reshape(-1)
    if b.size != nw or t.size != nw:
        raise ValueError("bot and top need one coefficient per mode")
    bb = np.ascontiguousarray(np.stack([b.real, b.imag], axis=1).reshape(-1))
    tt = np.ascontiguousarray(np.stack([t.real, t.imag], axis=1).reshape(-1))
    _check(load().qslab_set_walls(h, float(sigma_bot), float(sigma_top), nw,
                                  modes.ctypes.data if nw else None, bb.ctypes.data if nw else None,
                                  tt.ctypes.data if nw else None), "qslab_set_walls")


def qslab_set_rbe_sampler(h, kind, thin=1):
    """Random-batch k-sampler: QSLAB_SAMPLER_IID or QSLAB_SAMPLER_METROPOLIS
    (App. G) with downsampling rate thin."""
    _check(load().qslab_set_rbe_sampler(h, int(kind), int(thin)), "qslab_set_rbe_sampler")


def qslab_md_configure(h, dt, mass, gamma, kT, lj_eps, lj_sigma, wall_eps, wall_sigma, seed):
    _check(load().qslab_md_configure(h, float(dt), float(mass), float(gamma), float(kT),
                                     float(lj_eps), float(lj_sigma), float(wall_eps),
                                     float(wall_sigma), int(seed)), "qslab_md_configure")


def qslab_md_forces(h, N, pos_ptr, q_ptr, vel_ptr, force_ptr, energies_ptr, stream_ptr):
    _check(load().qslab_md_forces(h, N, pos_ptr, q_ptr, vel_ptr, force_ptr, energies_ptr,
                                  stream_ptr), "qslab_md_forces")


def qslab_md_step(h, N, pos_ptr, vel_ptr, q_ptr, force_ptr, nsteps, energies_ptr, stream_ptr):
    _check(load().qslab_md_step(h, N, pos_ptr, vel_ptr, q_ptr, force_ptr, int(nsteps),
                                energies_ptr, stream_ptr), "qslab_md_step")


def qslab_md_set_step(h, step):
    _check(load().qslab_md_set_step(h, int(step)), "qslab_md_set_step")


def qslab_md_get_step(h):
    v = ctypes.c_uint64(0)
    _check(load().qslab_md_get_step(h, ctypes.byref(v)), "qslab_md_get_step")
    return v.value


def qslab_clear_walls(h):
    _check(load().qslab_clear_walls(h), "qslab_clear_walls")


def qslab_compute_realspace(h, N, pos_ptr, q_ptr, energy_ptr, phi_ptr, force_ptr, stream_ptr):
    """Real-space part (Eq. 2.10) within the cut-off set by qslab_set_rcut."""
    _check(load().qslab_compute_realspace(h, N, pos_ptr, q_ptr, energy_ptr, phi_ptr, force_ptr,
                                          stream_ptr), "qslab_compute_realspace")


def qslab_get_sampled_modes(h, P, R=1):
    """(mx, my, weight) of the latest random-batch call: arrays of P (R = 1)
    or R x P, and the weight H/P (a float, or R of them)."""
    mxy = np.zeros(2 * P * R, np.int32)
    wt = np.zeros(R)
    _check(load().qslab_get_sampled_modes(h, mxy.ctypes.data, wt.ctypes.data),
           "qslab_get_sampled_modes")
    mx, my = mxy[0::2].copy(), mxy[1::2].copy()
    if R == 1:
        return mx, my, float(wt[0])
    return mx.reshape(R, P), my.reshape(R, P), wt


def qslab_get_rng_state(h):
    s = ctypes.c_uint64()
    c = ctypes.c_uint64()
    _check(load().qslab_get_rng_state(h, ctypes.addressof(s), ctypes.addressof(c)),
           "qslab_get_rng_state")
    return s.value, c.value


def qslab_set_rng_state(h, seed, counter):
    _check(load().qslab_set_rng_state(h, seed, counter), "qslab_set_rng_state")


def qslab_num_modes(h) -> int:
    r = load().qslab_num_modes(h)
    if r < 0:
        raise QslabError(r, "qslab_num_modes")
    return r


def qslab_last_status(h) -> int:
    return load().qslab_last_status(h)


def qslab_set_timing(h, enable: bool):
    _check(load().qslab_set_timing(h, int(bool(enable))), "qslab_set_timing")


TIMING_PHASES = ("sort", "modes", "aggregate", "carry", "recurrence", "kzero", "combine", "total")


def qslab_get_timings(h):
    """Per-phase milliseconds of the latest call and its kernel-launch count."""
    out = np.zeros(8)
    nl = ctypes.c_int()
    _check(load().qslab_get_timings(h, out.ctypes.data, ctypes.addressof(nl)), "qslab_get_timings")
    return dict(zip(TIMING_PHASES, out.tolist())), nl.value


def qslab_strerror(code: int) -> str:
    return load().qslab_strerror(code).decode()


# ---------------------------------------------------------------- wrapper


def qslab_debug_alloc_count() -> int:
    return int(load().qslab_debug_alloc_count())


def qslab_debug_fail_alloc(n: int):
    _check(load().qslab_debug_fail_alloc(int(n)), "qslab_debug_fail_alloc")


def qslab_debug_stall_sort(tile: int):
    _check(load().qslab_debug_stall_sort(int(tile)), "qslab_debug_stall_sort")


def kcut_for_tail(alpha: float, tail: float) -> float:
    """k_c with Gaussian tail e^{-k_c^2/(4 alpha^2)} = tail (Section 2.3)."""
    return 2.0 * alpha * math.sqrt(math.log(1.0 / tail))


class QSlab:
    """One configured context. Inputs/outputs are torch CUDA tensors."""

    def __init__(self, device: int = 0, precision: str = "fp64"):
        import torch
        self.torch = torch
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.np_dtype = np.float64 if precision == "fp64" else np.float32
        self.device = device
        self.h = qslab_create(device, _PREC[precision])
        self.P = 0
        self.last_R = 1

    def close(self):
        if self.h:
            qslab_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def configure(self, box, alpha, soe, kcut=None, rbe=None, tail=1e-8, rcut=None):
        """box=(Lx,Ly,Lz); soe=(s,w) or M; kcut (full k-sum) or rbe=(P, seed);
        rcut: the real-space cut-off for compute_realspace (optional)."""
        if isinstance(soe, int):
            soe = load_soe(soe)
        qslab_set_box(self.h, *map(float, box))
        self.box = tuple(map(float, box))
        qslab_set_alpha(self.h, float(alpha))
        qslab_set_soe(self.h, *soe)
        if rbe is not None:
            self.P = int(rbe[0])
            qslab_set_rbe(self.h, self.P, int(rbe[1]))
        else:
            qslab_set_kcut(self.h, float(kcut if kcut is not None else kcut_for_tail(alpha, tail)))
        if rcut is not None:
            qslab_set_rcut(self.h, float(rcut))
        return self

    def set_walls(self, sigma_bot, sigma_top, modes=None, bot=None, top=None):
        """Charged walls at z = 0 and z = Lz (see qslab_set_walls); None clears them."""
        if sigma_bot is None:
            qslab_clear_walls(self.h)
        else:
            qslab_set_walls(self.h, sigma_bot, sigma_top, modes, bot, top)
        return self

    def sampler(self, kind="iid", thin=1):
        """Random-batch k-sampler: "iid" (exact independent draws) or
        "metropolis" (the chain of App. G, keeping every thin-th state)."""
        k = {"iid": QSLAB_SAMPLER_IID, "metropolis": QSLAB_SAMPLER_METROPOLIS}[kind]
        qslab_set_rbe_sampler(self.h, k, thin)
        return self

    def tuning(self, chunk=0, modes_per_cta=0):
        qslab_set_tuning(self.h, chunk, modes_per_cta)
        return self

    def num_modes(self):
        return qslab_num_modes(self.h)

    def compute(self, pos, q, energy=None, phi=None, force=None, want_phi=True, want_force=True):
        """Returns (energy[1] float64, phi[N], force[N,3]) as CUDA tensors."""
        torch = self.torch
        dev = torch.device("cuda", self.device)
        if pos.device != dev or q.device != dev:
            raise ValueError("pos and q must be CUDA tensors on the context's device")
        pos = pos.to(self.dtype).contiguous()
        q = q.to(self.dtype).contiguous()
        N = q.shape[0]
        if energy is None:
            energy = torch.empty(1, dtype=torch.float64, device=dev)
        if phi is None and want_phi:
            phi = torch.empty(N, dtype=self.dtype, device=dev)
        if force is None and want_force:
            force = torch.empty((N, 3), dtype=self.dtype, device=dev)
        st = torch.cuda.current_stream(dev).cuda_stream
        qslab_compute(self.h, N, pos.data_ptr(), q.data_ptr(), energy.data_ptr(),
                      phi.data_ptr() if phi is not None else None,
                      force.data_ptr() if force is not None else None, st)
        self.last_R = 1
        return energy, phi, force

    def compute_batched(self, pos, q, offsets, boxes, energies=None, phi=None, force=None,
                        want_phi=True, want_force=True):
        """R slabs in one call: replica r owns rows offsets[r]:offsets[r+1] of
        pos (N x 3) and q (N), in the box boxes[r] = (Lx, Ly, Lz). offsets and
        boxes are host arrays. Returns (energies[R] float64, phi[N],
        force[N,3]) as CUDA tensors; passing the output tensors in reuses them
        (as a CUDA-graph replay needs)."""
        torch = self.torch
        dev = torch.device("cuda", self.device)
        if pos.device != dev or q.device != dev:
            raise ValueError("pos and q must be CUDA tensors on the context's device")
        if pos.dtype != self.dtype or q.dtype != self.dtype or not pos.is_contiguous() \
                or not q.is_contiguous():
            raise ValueError("pos and q must be contiguous tensors of the context's precision")
        off = np.ascontiguousarray(offsets, np.int64)
        R = off.shape[0] - 1
        N = q.shape[0]
        if int(off[-1]) != N:
            raise ValueError("offsets[-1] must equal the number of particles")
        if energies is None:
            energies = torch.empty(R, dtype=torch.float64, device=dev)
        if phi is None and want_phi:
            phi = torch.empty(N, dtype=self.dtype, device=dev)
        if force is None and want_force:
            force = torch.empty((N, 3), dtype=self.dtype, device=dev)
        st = torch.cuda.current_stream(dev).cuda_stream
        qslab_compute_batched(self.h, off, boxes, pos.data_ptr(), q.data_ptr(),
                              energies.data_ptr(),
                              phi.data_ptr() if phi is not None else None,
                              force.data_ptr() if force is not None else None, st)
        self.last_R = R
        return energies, phi, force

    def compute_virial(self, pos, q, want_phi=True):
        """Long-range energy, potentials, forces and the virial tensor
        W = (xx, yy, zz, xy, xz, yz) of the long-range energy (float64[6]), as
        CUDA tensors: (energy[1], phi[N] or None, force[N,3], virial[6])."""
        torch = self.torch
        dev = torch.device("cuda", self.device)
        if pos.device != dev or q.device != dev:
            raise ValueError("pos and q must be CUDA tensors on the context's device")
        pos = pos.to(self.dtype).contiguous()
        q = q.to(self.dtype).contiguous()
        N = q.shape[0]
        energy = torch.empty(1, dtype=torch.float64, device=dev)
        phi = torch.empty(N, dtype=self.dtype, device=dev) if want_phi else None
        force = torch.empty((N, 3), dtype=self.dtype, device=dev)
        virial = torch.empty(6, dtype=torch.float64, device=dev)
        st = torch.cuda.current_stream(dev).cuda_stream
        qslab_compute_virial(self.h, N, pos.data_ptr(), q.data_ptr(), energy.data_ptr(),
                             phi.data_ptr() if phi is not None else None, force.data_ptr(),
                             virial.data_ptr(), st)
        self.last_R = 1
        return energy, phi, force, virial

    def compute_energy(self, pos, q, energy=None):
        """Energy only (float64[1] CUDA tensor), from forward sums; the
        workspace is kept for adjoint()."""
        torch = self.torch
        dev = torch.device("cuda", self.device)
        if pos.device != dev or q.device != dev:
            raise ValueError("pos and q must be CUDA tensors on the context's device")
        pos = pos.to(self.dtype).contiguous()
        q = q.to(self.dtype).contiguous()
        N = q.shape[0]
        if energy is None:
            energy = torch.empty(1, dtype=torch.float64, device=dev)
        st = torch.cuda.current_stream(dev).cuda_stream
        qslab_compute_energy(self.h, N, pos.data_ptr(), q.data_ptr(), energy.data_ptr(), st)
        self.last_R = 1
        self._adjoint_n = N
        return energy

    def compute_batched_energy(self, pos, q, offsets, boxes, energies=None):
        """Energies of R slabs (float64[R]) from forward sums; the workspace
        is kept for adjoint()."""
        torch = self.torch
        dev = torch.device("cuda", self.device)
        if pos.dtype != self.dtype or q.dtype != self.dtype or not pos.is_contiguous() \
                or not q.is_contiguous() or pos.device != dev or q.device != dev:
            raise ValueError("pos and q must be contiguous CUDA tensors of the context's precision")
        off = np.ascontiguousarray(offsets, np.int64)
        R = off.shape[0] - 1
        if int(off[-1]) != q.shape[0]:
            raise ValueError("offsets[-1] must equal the number of particles")
        if energies is None:
            energies = torch.empty(R, dtype=torch.float64, device=dev)
        st = torch.cuda.current_stream(dev).cuda_stream
        qslab_compute_batched_energy(self.h, off, boxes, pos.data_ptr(), q.data_ptr(),
                                     energies.data_ptr(), st)
        self.last_R = R
        self._adjoint_n = q.shape[0]
        return energies

    def adjoint(self, phi=None, force=None):
        """(phi = dE/dq, F = -dE/dr) of the last energy-only call, in its
        particle order, as CUDA tensors."""
        torch = self.torch
        dev = torch.device("cuda", self.device)
        N = getattr(self, "_adjoint_n", None)
        if N is None:
            raise QslabError(-2, "qslab_compute_adjoint")
        if phi is None:
            phi = torch.empty(N, dtype=self.dtype, device=dev)
        if force is None:
            force = torch.empty((N, 3), dtype=self.dtype, device=dev)
        st = torch.cuda.current_stream(dev).cuda_stream
        qslab_compute_adjoint(self.h, phi.data_ptr(), force.data_ptr(), st)
        return phi, force

    def compute_batched_virial(self, pos, q, offsets, boxes):
        """compute_batched() plus each replica's virial: returns (energies[R],
        phi[N], force[N,3], virial[R,6]) as CUDA tensors."""
        torch = self.torch
        dev = torch.device("cuda", self.device)
        if pos.dtype != self.dtype or q.dtype != self.dtype or not pos.is_contiguous() \
                or not q.is_contiguous() or pos.device != dev or q.device != dev:
            raise ValueError("pos and q must be contiguous CUDA tensors of the context's precision")
        off = np.ascontiguousarray(offsets, np.int64)
        R = off.shape[0] - 1
        N = q.shape[0]
        if int(off[-1]) != N:
            raise ValueError("offsets[-1] must equal the number of particles")
        energies = torch.empty(R, dtype=torch.float64, device=dev)
        phi = torch.empty(N, dtype=self.dtype, device=dev)
        force = torch.empty((N, 3), dtype=self.dtype, device=dev)
        virial = torch.empty((R, 6), dtype=torch.float64, device=dev)
        st = torch.cuda.current_stream(dev).cuda_stream
        qslab_compute_batched_virial(self.h, off, boxes, pos.data_ptr(), q.data_ptr(),
                                     energies.data_ptr(), phi.data_ptr(), force.data_ptr(),
                                     virial.data_ptr(), st)
        self.last_R = R
        return energies, phi, force, virial

    def compute_realspace_virial(self, pos, q):
        """Real-space part and its pair virial: (energy[1], phi[N], force[N,3],
        virial[6]) as CUDA tensors."""
        torch = self.torch
        dev = torch.device("cuda", self.device)
        if pos.device != dev or q.device != dev:
            raise ValueError("pos and q must be CUDA tensors on the context's device")
        pos = pos.to(self.dtype).contiguous()
        q = q.to(self.dtype).contiguous()
        N = q.shape[0]
        energy = torch.empty(1, dtype=torch.float64, device=dev)
        phi = torch.empty(N, dtype=self.dtype, device=dev)
        force = torch.empty((N, 3), dtype=self.dtype, device=dev)
        virial = torch.empty(6, dtype=torch.float64, device=dev)
        st = torch.cuda.current_stream(dev).cuda_stream
        qslab_compute_realspace_virial(self.h, N, pos.data_ptr(), q.data_ptr(), energy.data_ptr(),
                                       phi.data_ptr(), force.data_ptr(), virial.data_ptr(), st)
        return energy, phi, force, virial

    def compute_realspace(self, pos, q, energy=None, phi=None, force=None, want_phi=True,
                          want_force=True):
        """Real-space part: (energy[1] float64, phi[N], force[N,3]) as CUDA tensors."""
        torch = self.torch
        dev = torch.device("cuda", self.device)
        if pos.device != dev or q.device != dev:
            raise ValueError("pos and q must be CUDA tensors on the context's device")
        pos = pos.to(self.dtype).contiguous()
        q = q.to(self.dtype).contiguous()
        N = q.shape[0]
        if energy is None:
            energy = torch.empty(1, dtype=torch.float64, device=dev)
        if phi is None and want_phi:
            phi = torch.empty(N, dtype=self.dtype, device=dev)
        if force is None and want_force:
            force = torch.empty((N, 3), dtype=self.dtype, device=dev)
        st = torch.cuda.current_stream(dev).cuda_stream
        qslab_compute_realspace(self.h, N, pos.data_ptr(), q.data_ptr(), energy.data_ptr(),
                                phi.data_ptr() if phi is not None else None,
                                force.data_ptr() if force is not None else None, st)
        return energy, phi, force

    def md_configure(self, dt, mass=1.0, gamma=1.0, kT=1.0, lj=(1.0, 1.0), wall=(1.0, 0.5),
                     seed=0):
        """Langevin dynamics (BAOAB): lj=(eps, sigma) between particles and
        wall=(eps, sigma) at both walls, or None to leave a term out."""
        lj = lj or (0.0, 0.0)
        wall = wall or (0.0, 0.0)
        qslab_md_configure(self.h, dt, mass, gamma, kT, lj[0], lj[1], wall[0], wall[1], seed)
        return self

    def _md_check(self, *ts):
        dev = self.torch.device("cuda", self.device)
        for t in ts:
            if t is not None and (t.device != dev or t.dtype != self.dtype or not t.is_contiguous()):
                raise ValueError("MD arrays must be contiguous CUDA tensors of the context's dtype")

    def md_forces(self, pos, q, vel=None, force=None, energies=None):
        """Total force at pos; returns (force[N,3], energies[4]): long range,
        real space + LJ pairs, LJ walls, kinetic."""
        torch = self.torch
        dev = torch.device("cuda", self.device)
        N = q.shape[0]
        if force is None:
            force = torch.empty((N, 3), dtype=self.dtype, device=dev)
        if energies is None:
            energies = torch.empty(4, dtype=torch.float64, device=dev)
        self._md_check(pos, q, vel, force)
        st = torch.cuda.current_stream(dev).cuda_stream
        qslab_md_forces(self.h, N, pos.data_ptr(), q.data_ptr(),
                        vel.data_ptr() if vel is not None else None, force.data_ptr(),
                        energies.data_ptr(), st)
        return force, energies

    def md_step(self, pos, vel, q, force, nsteps=1, energies=None):
        """nsteps BAOAB steps in place (pos, vel, force); returns energies[4]."""
        torch = self.torch
        dev = torch.device("cuda", self.device)
        if energies is None:
            energies = torch.empty(4, dtype=torch.float64, device=dev)
        self._md_check(pos, vel, q, force)
        st = torch.cuda.current_stream(dev).cuda_stream
        qslab_md_step(self.h, q.shape[0], pos.data_ptr(), vel.data_ptr(), q.data_ptr(),
                      force.data_ptr(), nsteps, energies.data_ptr(), st)
        return energies

    def compute_host(self, pos, q, stream=None):
        """Host numpy in, host numpy out, through qslab_compute_host."""
        pos = np.ascontiguousarray(pos, self.np_dtype)
        q = np.ascontiguousarray(q, self.np_dtype)
        N = q.shape[0]
        e = np.zeros(1)
        phi = np.zeros(N, self.np_dtype)
        F = np.zeros((N, 3), self.np_dtype)
        qslab_compute_host(self.h, N, pos.ctypes.data, q.ctypes.data, e.ctypes.data,
                           phi.ctypes.data, F.ctypes.data, stream)
        return float(e[0]), phi, F

    def autotune(self, pos, q, offsets=None, boxes=None, reps=3):
        """Pick the launch shape (chunk length, modes per CTA) by timing the
        candidates on these inputs; for a single slab leave offsets and boxes
        None. Returns the chosen (chunk, modes_per_cta)."""
        torch = self.torch
        dev = torch.device("cuda", self.device)
        N = q.shape[0]
        if offsets is None:
            offsets = np.array([0, N], np.int64)
            boxes = np.array([self.box], np.float64)
        st = torch.cuda.current_stream(dev).cuda_stream
        return qslab_autotune(self.h, offsets, boxes, pos.data_ptr(), q.data_ptr(), st, reps)

    def status(self):
        return qslab_last_status(self.h)

    def set_neutrality_tol(self, tol):
        """Relative neutrality tolerance; a negative value turns the check off."""
        qslab_set_neutrality_tol(self.h, float(tol))
        return self

    def check(self):
        rc = qslab_last_status(self.h)
        if rc != 0:
            raise QslabError(rc, "device status")

    def sampled_modes(self):
        return qslab_get_sampled_modes(self.h, self.P, self.last_R)

    def rng_state(self):
        return qslab_get_rng_state(self.h)

    def set_rng_state(self, seed, counter):
        qslab_set_rng_state(self.h, seed, counter)


class GraphedBatch:
    """qslab_compute_batched captured once in a CUDA graph and replayed.

    The inputs pos and q (CUDA tensors of the context's precision) are read
    in place at every replay: write new coordinates into them, then call
    replay(). Outputs land in self.energies, self.phi and self.force. A
    random-batch context draws a fresh sample at every replay (its counter
    lives on the device). The replica layout (offsets, boxes) is fixed by the
    capture."""

    def __init__(self, slab: QSlab, pos, q, offsets, boxes, warmup: int = 1):
        import torch
        self.slab = slab
        self.pos, self.q = pos, q
        self.offsets = np.ascontiguousarray(offsets, np.int64)
        self.boxes = np.ascontiguousarray(boxes, np.float64)
        dev = pos.device
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            # sizes the context (tables, workspace) so that the captured call
            # only issues stream-ordered work
            out = slab.compute_batched(pos, q, self.offsets, self.boxes)
            for _ in range(max(0, warmup - 1)):
                slab.compute_batched(pos, q, self.offsets, self.boxes, *out)
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize(dev)
        self.energies, self.phi, self.force = out
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            slab.compute_batched(pos, q, self.offsets, self.boxes, self.energies, self.phi,
                                 self.force)

    def replay(self):
        self.graph.replay()
        return self.energies, self.phi, self.force


class GraphedMD:
    """nsteps of qslab_md_step captured once in a CUDA graph. pos, vel and
    force are updated in place at every replay; the noise and random-batch
    counters live on the device, so replays continue the trajectory."""

    def __init__(self, slab: QSlab, pos, vel, q, force, nsteps: int = 1):
        import torch
        self.slab, self.pos, self.vel, self.q, self.force = slab, pos, vel, q, force
        self.nsteps = int(nsteps)
        dev = pos.device
        self.energies = torch.empty(4, dtype=torch.float64, device=dev)
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            # sizes every buffer, so that the captured call only issues
            # stream-ordered work (this warm-up advances the trajectory)
            slab.md_step(pos, vel, q, force, self.nsteps, self.energies)
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize(dev)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            slab.md_step(pos, vel, q, force, self.nsteps, self.energies)

    def replay(self):
        self.graph.replay()
        return self.energies


def _autograd():
    import torch

    class SlabEnergy(torch.autograd.Function):
        """E(pos, q) with the exact adjoint: dE/dpos = -F, dE/dq = phi.

        adjoint=False: the forward runs the full call and keeps phi and F.
        adjoint=True: the forward runs the energy-only call (forward sums);
        the backward runs qslab_compute_adjoint, the bidirectional scans over
        the sorted order the forward left in the workspace (nothing N x K is
        stored). No other call may use the context between the two."""

        @staticmethod
        def forward(ctx, pos, q, slab: QSlab, adjoint: bool):
            ctx.dtypes = (pos.dtype, q.dtype)
            ctx.adjoint = adjoint
            ctx.slab = slab
            if adjoint:
                e = slab.compute_energy(pos.detach(), q.detach())
                return e[0].to(pos.dtype)
            e, phi, F = slab.compute(pos.detach(), q.detach())
            ctx.save_for_backward(phi, F)
            return e[0].to(pos.dtype)

        @staticmethod
        def backward(ctx, gE):
            if ctx.adjoint:
                phi, F = ctx.slab.adjoint()
            else:
                phi, F = ctx.saved_tensors
            gpos = (-gE * F).to(ctx.dtypes[0])
            gq = (gE * phi).to(ctx.dtypes[1])
            return gpos, gq, None, None

    return SlabEnergy


def slab_energy(pos, q, slab: QSlab, adjoint: bool = False):
    """Differentiable long-range energy (torch autograd); adjoint=True
    computes only the energy in the forward and the gradient in the
    backward (see SlabEnergy)."""
    return _autograd().apply(pos, q, slab, adjoint)
