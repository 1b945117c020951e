"""Thin Python binding of the C ABI in include/nep.h (argument marshalling only).

Every step of the evaluation runs in the CUDA library libnep_gb300.so; this module
only converts arrays to pointers.  Host arrays are numpy; device arrays are torch
CUDA tensors (torch supplies device memory and streams).  If the library is not
built, load() raises -- there is no CPU fallback.

Module-level functions carry the C names (nep_create, nep_compute, nep_md_step,
nep_neighbors, ...); `Model` wraps a handle for convenience.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

NEP_OK = 0
NEP_ERR_ARG = -1
NEP_ERR_OOM = -2
NEP_ERR_NEIGHBOR_OVERFLOW = -3
NEP_ERR_BOX_TOO_SMALL = -4
NEP_ERR_TIMEOUT = -5
NEP_ERR_CUDA = -6
NEP_ERR_UNSUPPORTED = -7
NEP_FP64 = 0
NEP_FP32 = 1
NEP_FP32_BF16 = 2
PRECISIONS = {"fp64": NEP_FP64, "fp32": NEP_FP32, "bf16": NEP_FP32_BF16}
NEP_HOST = 0
NEP_DEVICE = 1

EXPORTED = ["nep_version", "nep_error_string", "nep_last_error", "nep_create", "nep_supported_shape",
            "nep_destroy", "nep_compute", "nep_md_step", "nep_scale_positions", "nep_neighbors",
            "nep_get_capacity", "nep_set_capacity", "nep_sync", "nep_set_timing", "nep_get_timing",
            "nep_compute_static", "nep_compute_batch", "nep_md_step_nvt", "nep_cg_map",
            "nep_virial_correction", "nep_autotune", "nep_set_tuning", "nep_get_tuning", "nep_md_step_hnemd",
            "nep_request_workspace", "nep_workspace_bytes", "nep_host_alloc", "nep_host_free"]

_lib = None


class NepError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = f"{where}: {_lib.nep_error_string(code).decode()} ({code})"
        detail = _lib.nep_last_error().decode()
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libnep_gb300.so; raise if it is not built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if build_if_missing:
        _build.build()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run paper_2603_01234_gb300/build.py)")
    lib = C.CDLL(path)
    i, d, p = C.c_int, C.c_double, C.c_void_p
    lib.nep_version.restype = i
    lib.nep_error_string.argtypes = [i]
    lib.nep_error_string.restype = C.c_char_p
    lib.nep_last_error.restype = C.c_char_p
    lib.nep_create.argtypes = [C.POINTER(p), i, p, p, i, i, i, i, i, i, i, i, p, p, p, p, p, p, i, i]
    lib.nep_create.restype = i
    lib.nep_supported_shape.argtypes = [i] * 7
    lib.nep_supported_shape.restype = i
    lib.nep_destroy.argtypes = [p]
    lib.nep_destroy.restype = i
    lib.nep_compute.argtypes = [p, i, p, p, p, p, i, p, p, p, p, p, p]
    lib.nep_compute.restype = i
    lib.nep_md_step.argtypes = [p, i, p, p, p, p, p, p, p, i, i, d, i, p, i, p]
    lib.nep_md_step.restype = i
    lib.nep_scale_positions.argtypes = [p, i, p, p, i, p]
    lib.nep_scale_positions.restype = i
    lib.nep_neighbors.argtypes = [p, i, p, p, p, p, i, i, p, p, p]
    lib.nep_neighbors.restype = i
    lib.nep_get_capacity.argtypes = [p, C.POINTER(i), C.POINTER(i)]
    lib.nep_get_capacity.restype = i
    lib.nep_set_capacity.argtypes = [p, i, i]
    lib.nep_set_capacity.restype = i
    lib.nep_sync.argtypes = [p]
    lib.nep_sync.restype = i
    lib.nep_set_timing.argtypes = [p, i]
    lib.nep_set_timing.restype = i
    lib.nep_get_timing.argtypes = [p, p, C.POINTER(C.c_longlong)]
    lib.nep_get_timing.restype = i
    lib.nep_compute_static.argtypes = [p, i, p, p, p, p, p, p, p, p, p, p]
    lib.nep_compute_static.restype = i
    lib.nep_compute_batch.argtypes = [p, i, i, p, p, p, p, p, p, i, p, p, p, p, p, p]
    lib.nep_compute_batch.restype = i
    lib.nep_md_step_nvt.argtypes = [p, i, p, p, p, p, p, p, p, i, i, d, d, d, p, i, p, i, p]
    lib.nep_md_step_nvt.restype = i
    lib.nep_md_step_hnemd.argtypes = [p, i, p, p, p, p, p, p, p, i, i, d, p, d, d, p, i, p, p, i, p]
    lib.nep_md_step_hnemd.restype = i
    lib.nep_cg_map.argtypes = [p, i, p, p, i, p, p, p, p, p, p, i, i, p, p, p, p]
    lib.nep_cg_map.restype = i
    lib.nep_virial_correction.argtypes = [p, i, i, d]
    lib.nep_virial_correction.restype = i
    lib.nep_autotune.argtypes = [p, i, p, p, p, p, i, p, C.POINTER(i), C.POINTER(i), C.POINTER(i)]
    lib.nep_autotune.restype = i
    lib.nep_set_tuning.argtypes = [p, i, i, i, i]
    lib.nep_set_tuning.restype = i
    lib.nep_get_tuning.argtypes = [p, C.POINTER(i), C.POINTER(i), C.POINTER(i)]
    lib.nep_get_tuning.restype = i
    lib.nep_request_workspace.argtypes = [p, i, i, i, p, p, C.POINTER(C.c_size_t)]
    lib.nep_request_workspace.restype = i
    lib.nep_workspace_bytes.argtypes = [p, C.POINTER(C.c_size_t)]
    lib.nep_workspace_bytes.restype = i
    lib.nep_host_alloc.argtypes = [C.c_size_t, C.POINTER(p)]
    lib.nep_host_alloc.restype = i
    lib.nep_host_free.argtypes = [p]
    lib.nep_host_free.restype = i
    _lib = lib
    return lib


def _check(code, where):
    if code != NEP_OK:
        raise NepError(code, where)


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """Pointer of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if _is_torch(x):
        return C.c_void_p(x.data_ptr())
    return x.ctypes.data_as(C.c_void_p)


def _stream_of(x, stream):
    if stream is not None:
        return C.c_void_p(stream)
    if x is not None and _is_torch(x) and x.is_cuda:
        import torch
        return C.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
    return None


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---- C-named functions ---------------------------------------------------------
def nep_version():
    return load().nep_version()


def nep_supported_shape(n_desc_radial, n_desc_angular, n_basis_radial, n_basis_angular, l_max, l_max_4b=0,
                        l_max_5b=0):
    return bool(load().nep_supported_shape(n_desc_radial, n_desc_angular, n_basis_radial, n_basis_angular, l_max,
                                           l_max_4b, l_max_5b))


def nep_create(params, precision=NEP_FP32, device=0):
    """params: an inputs.ModelParams.  Returns an opaque handle (c_void_p)."""
    lib = load()
    h = C.c_void_p()
    T, H = params.n_types, params.hidden
    if np.size(params.w0) != T * H * params.n_des:
        raise ValueError(f"w0 has {np.size(params.w0)} entries, expected [T][H][N_des] = {T * H * params.n_des}")
    arrs = [_host(params.rc_radial, np.float64), _host(params.rc_angular, np.float64),
            _host(params.c_radial, np.float64), _host(params.c_angular, np.float64),
            _host(params.w0, np.float64), _host(params.b0, np.float64), _host(params.w1, np.float64),
            _host(params.b1, np.float64)]
    _check(lib.nep_create(C.byref(h), params.n_types, _ptr(arrs[0]), _ptr(arrs[1]), params.n_basis_radial,
                          params.n_basis_angular, params.n_desc_radial, params.n_desc_angular, params.l_max,
                          int(getattr(params, "l_max_4b", 0)), int(getattr(params, "l_max_5b", 0)),
                          params.hidden, *[_ptr(a) for a in arrs[2:]], int(precision), int(device)), "nep_create")
    return h


def nep_destroy(h):
    if h:
        _check(load().nep_destroy(h), "nep_destroy")


def nep_compute(h, types, pos, box, pbc, energy_total=None, virial_total=None, site_energy=None, force=None,
                virial=None, stream=None):
    """All arrays numpy (host) or all torch CUDA tensors (device); box/pbc host."""
    mem = NEP_DEVICE if _is_torch(pos) and pos.is_cuda else NEP_HOST
    n = int(types.shape[0])
    box = _host(box, np.float64)
    pbc = _host(pbc, np.int32)
    _check(load().nep_compute(h, n, _ptr(types), _ptr(pos), _ptr(box), _ptr(pbc), mem, _stream_of(pos, stream),
                              _ptr(energy_total), _ptr(virial_total), _ptr(site_energy), _ptr(force), _ptr(virial)),
           "nep_compute")


def nep_compute_static(h, types, pos, box, pbc, energy_total=None, virial_total=None, site_energy=None,
                       force=None, virial=None, stream=None):
    """Allocation-free evaluation: torch CUDA tensors only (device memory), n <= 4096."""
    n = int(types.shape[0])
    box = _host(box, np.float64)
    pbc = _host(pbc, np.int32)
    _check(load().nep_compute_static(h, n, _ptr(types), _ptr(pos), _ptr(box), _ptr(pbc), _stream_of(pos, stream),
                                     _ptr(energy_total), _ptr(virial_total), _ptr(site_energy), _ptr(force),
                                     _ptr(virial)), "nep_compute_static")


def nep_compute_batch(handles, req_n, req_model, req_box, req_pbc, types, pos, energy=None, virial_total=None,
                      site_energy=None, force=None, virial=None, stream=None):
    """Batched evaluation.  handles: list of model handles; arrays concatenated per
    request (numpy for host memory, torch CUDA tensors for device memory)."""
    mem = NEP_DEVICE if _is_torch(pos) and pos.is_cuda else NEP_HOST
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    req_n = _host(req_n, np.int32)
    req_model = _host(req_model, np.int32)
    req_box = _host(req_box, np.float64)
    req_pbc = _host(req_pbc, np.int32)
    _check(load().nep_compute_batch(C.cast(arr, C.c_void_p), len(handles), int(req_n.size), _ptr(req_n),
                                    _ptr(req_model), _ptr(req_box), _ptr(req_pbc), _ptr(types), _ptr(pos), mem,
                                    _stream_of(pos, stream), _ptr(energy), _ptr(virial_total), _ptr(site_energy),
                                    _ptr(force), _ptr(virial)), "nep_compute_batch")


def pack_requests(systems):
    """Concatenate systems into the batch layout: (req_n, req_box, req_pbc, types, pos)
    with pos as per-request [3][n_r] blocks."""
    req_n = np.array([s.n for s in systems], np.int32)
    req_box = np.array([s.box for s in systems], np.float64)
    req_pbc = np.array([s.pbc for s in systems], np.int32)
    types = np.concatenate([s.types for s in systems]).astype(np.int32)
    pos = np.concatenate([np.ascontiguousarray(s.pos, dtype=np.float64).reshape(-1) for s in systems])
    return req_n, req_box, req_pbc, types, pos


def unpack_blocks(arr, req_n, width):
    """Split a concatenated per-request [width][n_r] block array into a list."""
    out, o = [], 0
    for n in req_n:
        out.append(arr[o:o + width * n].reshape(width, n))
        o += width * n
    return out


def nep_md_step(h, types, masses, box, pbc, pos, vel, force, forces_valid, n_steps, dt_fs, sample_every=0,
                thermo=None, stream=None):
    mem = NEP_DEVICE if _is_torch(pos) and pos.is_cuda else NEP_HOST
    n = int(types.shape[0])
    masses = _host(masses, np.float64)
    box = _host(box, np.float64)
    pbc = _host(pbc, np.int32)
    _check(load().nep_md_step(h, n, _ptr(types), _ptr(masses), _ptr(box), _ptr(pbc), _ptr(pos), _ptr(vel),
                              _ptr(force), int(forces_valid), int(n_steps), float(dt_fs), int(sample_every),
                              _ptr(thermo), mem, _stream_of(pos, stream)), "nep_md_step")


STAGES = ["kick_drift", "cell_build", "neighbor_lists", "descriptor_network", "force_virial", "kick_sample"]


def nep_set_timing(h, enable):
    _check(load().nep_set_timing(h, int(enable)), "nep_set_timing")


def nep_get_timing(h):
    """Returns ({stage: summed ms}, steps)."""
    ms = np.zeros(6)
    steps = C.c_longlong()
    _check(load().nep_get_timing(h, _ptr(ms), C.byref(steps)), "nep_get_timing")
    return dict(zip(STAGES, ms.tolist())), steps.value


def nep_md_step_nvt(h, types, masses, box, pbc, pos, vel, force, forces_valid, n_steps, dt_fs, temperature_K,
                    tau_fs, noise, sample_every=0, thermo=None, stream=None):
    mem = NEP_DEVICE if _is_torch(pos) and pos.is_cuda else NEP_HOST
    n = int(types.shape[0])
    masses = _host(masses, np.float64)
    box = _host(box, np.float64)
    pbc = _host(pbc, np.int32)
    noise = _host(noise, np.float64)
    _check(load().nep_md_step_nvt(h, n, _ptr(types), _ptr(masses), _ptr(box), _ptr(pbc), _ptr(pos), _ptr(vel),
                                  _ptr(force), int(forces_valid), int(n_steps), float(dt_fs), float(temperature_K),
                                  float(tau_fs), _ptr(noise), int(sample_every), _ptr(thermo), mem,
                                  _stream_of(pos, stream)), "nep_md_step_nvt")


def nep_md_step_hnemd(h, types, masses, box, pbc, pos, vel, force, forces_valid, n_steps, dt_fs, fe,
                      temperature_K=0.0, tau_fs=1.0, noise=None, sample_every=0, thermo=None, heat=None, stream=None):
    """HNEMD steps (driving force fe[3], optional thermostat noise); heat [samples][6]
    receives the interval-averaged (J_pot, J_kin)."""
    mem = NEP_DEVICE if _is_torch(pos) and pos.is_cuda else NEP_HOST
    n = int(types.shape[0])
    masses = _host(masses, np.float64)
    box = _host(box, np.float64)
    pbc = _host(pbc, np.int32)
    fe = _host(fe, np.float64)
    noise = None if noise is None else _host(noise, np.float64)
    _check(load().nep_md_step_hnemd(h, n, _ptr(types), _ptr(masses), _ptr(box), _ptr(pbc), _ptr(pos), _ptr(vel),
                                    _ptr(force), int(forces_valid), int(n_steps), float(dt_fs), _ptr(fe),
                                    float(temperature_K), float(tau_fs), _ptr(noise), int(sample_every),
                                    _ptr(thermo), _ptr(heat), mem, _stream_of(pos, stream)), "nep_md_step_hnemd")


def bussi_noise(n_steps, n_particles, seed):
    """Random numbers of the thermostat: [n_steps][2] = (R1 ~ N(0,1), chi^2(3n - 4))."""
    rng = np.random.default_rng(seed)
    out = np.empty((n_steps, 2))
    out[:, 0] = rng.standard_normal(n_steps)
    out[:, 1] = rng.chisquare(3 * n_particles - 4, size=n_steps)
    return out


def nep_cg_map(h, group_start, group_atoms, atom_mass, atom_pos, box, pbc, atom_force=None, atom_virial=None,
               accumulate=False, bead_pos=None, bead_force=None, bead_virial=None, stream=None):
    """Bead positions / forces / virials of CSR atom groups (Eq. 9, 12, 14).  Host
    numpy arrays or device torch tensors; returns the outputs it was given or made."""
    dev = _is_torch(atom_pos) and atom_pos.is_cuda
    mem = NEP_DEVICE if dev else NEP_HOST
    n_cg = int(group_start.shape[0]) - 1
    n_aa = int(atom_mass.shape[0])
    if not dev:
        group_start, group_atoms = _host(group_start, np.int32), _host(group_atoms, np.int32)
        atom_mass, atom_pos = _host(atom_mass, np.float64), _host(atom_pos, np.float64)
        atom_force = None if atom_force is None else _host(atom_force, np.float64)
        atom_virial = None if atom_virial is None else _host(atom_virial, np.float64)
        if bead_pos is None:
            bead_pos = np.zeros((3, n_cg))
        if bead_force is None and atom_force is not None:
            bead_force = np.zeros((3, n_cg))
        if bead_virial is None and atom_virial is not None:
            bead_virial = np.zeros((9, n_cg))
    _check(load().nep_cg_map(h, n_cg, _ptr(group_start), _ptr(group_atoms), n_aa, _ptr(atom_mass), _ptr(atom_pos),
                             _ptr(atom_force), _ptr(atom_virial), _ptr(_host(box, np.float64)),
                             _ptr(_host(pbc, np.int32)), int(accumulate), mem, _stream_of(atom_pos, stream),
                             _ptr(bead_pos), _ptr(bead_force), _ptr(bead_virial)), "nep_cg_map")
    return bead_pos, bead_force, bead_virial


def nep_virial_correction(virial, n_atoms, n_beads, temperature_K):
    v = _host(virial, np.float64).copy()
    _check(load().nep_virial_correction(_ptr(v), int(n_atoms), int(n_beads), float(temperature_K)),
           "nep_virial_correction")
    return v


def nep_autotune(h, types, pos, box, pbc, stream=None):
    """Tune the kernel variants on this configuration; returns (mb_desc, mb_force, chunk)."""
    mem = NEP_DEVICE if _is_torch(pos) and pos.is_cuda else NEP_HOST
    if mem == NEP_HOST:
        types, pos = _host(types, np.int32), _host(pos, np.float64)
    a, b, c = C.c_int(), C.c_int(), C.c_int()
    _check(load().nep_autotune(h, int(types.shape[0]), _ptr(types), _ptr(pos), _ptr(_host(box, np.float64)),
                               _ptr(_host(pbc, np.int32)), mem, _stream_of(pos, stream), C.byref(a), C.byref(b),
                               C.byref(c)),
           "nep_autotune")
    return a.value, b.value, c.value


def nep_set_tuning(h, autotune, mb_desc, mb_force, chunk=4):
    _check(load().nep_set_tuning(h, int(autotune), int(mb_desc), int(mb_force), int(chunk)), "nep_set_tuning")


def nep_get_tuning(h):
    """The kernel variants in use: (mb_desc, mb_force, chunk)."""
    a, b, c = C.c_int(), C.c_int(), C.c_int()
    _check(load().nep_get_tuning(h, C.byref(a), C.byref(b), C.byref(c)), "nep_get_tuning")
    return a.value, b.value, c.value


def nep_request_workspace(handles, model, n, box, pbc):
    """Device bytes one request (of handles[model], n particles in box) adds to a
    batch evaluated on handles[0]'s workspace."""
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    out = C.c_size_t()
    _check(load().nep_request_workspace(C.cast(arr, C.c_void_p), len(handles), int(model), int(n),
                                        _ptr(_host(box, np.float64)), _ptr(_host(pbc, np.int32)), C.byref(out)),
           "nep_request_workspace")
    return out.value


def nep_workspace_bytes(h):
    out = C.c_size_t()
    _check(load().nep_workspace_bytes(h, C.byref(out)), "nep_workspace_bytes")
    return out.value


class PinnedBuffer:
    """Page-locked host memory from nep_host_alloc, viewed as numpy arrays."""

    def __init__(self, nbytes):
        self.nbytes = int(nbytes)
        ptr = C.c_void_p()
        _check(load().nep_host_alloc(self.nbytes, C.byref(ptr)), "nep_host_alloc")
        self.ptr = ptr.value
        self._raw = (C.c_ubyte * self.nbytes).from_address(self.ptr)

    def view(self, offset, count, dtype):
        dtype = np.dtype(dtype)
        return np.frombuffer(self._raw, dtype=dtype, count=count, offset=offset)

    def close(self):
        if self.ptr:
            self._raw = None
            load().nep_host_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nep_sync(h):
    _check(load().nep_sync(h), "nep_sync")


def nep_scale_positions(h, pos, scale, stream=None):
    mem = NEP_DEVICE if _is_torch(pos) and pos.is_cuda else NEP_HOST
    n = int(pos.shape[1])
    scale = _host(scale, np.float64)
    _check(load().nep_scale_positions(h, n, _ptr(pos), _ptr(scale), mem, _stream_of(pos, stream)),
           "nep_scale_positions")


def nep_neighbors(h, types, pos, box, pbc, kind, capacity):
    """Host arrays.  Returns (count[n], j[n][cap], shift[n][cap][3])."""
    n = int(types.shape[0])
    types = _host(types, np.int32)
    pos = _host(pos, np.float64)
    box = _host(box, np.float64)
    pbc = _host(pbc, np.int32)
    cnt = np.zeros(n, np.int32)
    j = np.full((n, capacity), -1, np.int32)
    sh = np.zeros((n, capacity, 3), np.int32)
    _check(load().nep_neighbors(h, n, _ptr(types), _ptr(pos), _ptr(box), _ptr(pbc), int(kind), int(capacity),
                                _ptr(cnt), _ptr(j), _ptr(sh)), "nep_neighbors")
    return cnt, j, sh


def nep_get_capacity(h):
    r, a = C.c_int(), C.c_int()
    _check(load().nep_get_capacity(h, C.byref(r), C.byref(a)), "nep_get_capacity")
    return r.value, a.value


def nep_set_capacity(h, radial, angular):
    _check(load().nep_set_capacity(h, int(radial), int(angular)), "nep_set_capacity")


# ---- convenience wrapper -------------------------------------------------------
class Model:
    """A model handle.  precision: "fp32", "fp64" or "bf16" (FP32 with BF16
    hidden-layer weights W0 and the hidden layer's products on tensor cores)."""

    def __init__(self, params, precision="fp32", device=0):
        self.params = params
        self.precision = precision
        self.device = device
        self.h = nep_create(params, PRECISIONS[precision], device)

    def close(self):
        if self.h:
            nep_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def compute(self, system_or_types, pos=None, box=None, pbc=None, stream=None):
        """Host evaluation; returns dict(energy, virial_total, site_energy, force, virial)."""
        if pos is None:
            s = system_or_types
            types, pos, box, pbc = s.types, s.pos, s.box, s.pbc
        else:
            types = system_or_types
        n = int(types.shape[0])
        e = np.zeros(1)
        wt = np.zeros(9)
        U = np.zeros(n)
        F = np.zeros((3, n))
        W = np.zeros((9, n))
        nep_compute(self.h, _host(types, np.int32), _host(pos, np.float64), box, pbc, e, wt, U, F, W, stream=stream)
        return {"energy": float(e[0]), "virial_total": wt, "site_energy": U, "force": F, "virial": W}

    def compute_device(self, types, pos, box, pbc, out=None, stream=None):
        """Device evaluation on torch CUDA tensors; returns dict of tensors."""
        import torch
        n = int(types.shape[0])
        dev = pos.device
        if out is None:
            out = {"energy": torch.zeros(1, dtype=torch.float64, device=dev),
                   "virial_total": torch.zeros(9, dtype=torch.float64, device=dev),
                   "site_energy": torch.zeros(n, dtype=torch.float64, device=dev),
                   "force": torch.zeros(3, n, dtype=torch.float64, device=dev),
                   "virial": torch.zeros(9, n, dtype=torch.float64, device=dev)}
        nep_compute(self.h, types, pos, box, pbc, out["energy"], out["virial_total"], out["site_energy"],
                    out["force"], out["virial"], stream=stream)
        return out

    def neighbors(self, system, kind=0, capacity=None):
        cap = capacity or max(nep_get_capacity(self.h)) or 256
        return nep_neighbors(self.h, system.types, system.pos, system.box, system.pbc, kind, max(cap, 8))
