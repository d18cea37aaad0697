"""Thin Python binding of libcamp.so (C ABI in include/camp.h).

Argument marshalling only: every step of the solve runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcamp.so")

VARIANT_MIXED = 0
VARIANT_FP64 = 1
NSTATS = 5  # steps, Newton iterations, J/LU setups, error-test failures, sum of orders

CELL_STATUS = {0: "ok", 1: "max_steps", 2: "error_test", 3: "newton", 4: "singular", 5: "nonfinite"}

_lib = None


class CampError(RuntimeError):
    pass


class MechInfo(ctypes.Structure):
    _fields_ = [("n_species", ctypes.c_int32), ("n_rxn", ctypes.c_int32),
                ("n_env", ctypes.c_int32), ("n_sections", ctypes.c_int32),
                ("nnz_jac", ctypes.c_int32), ("nnz_lu", ctypes.c_int32),
                ("rxn_map_len", ctypes.c_int32), ("dense_block", ctypes.c_int32),
                ("lu_storage", ctypes.c_int32), ("smem_per_cell_mixed", ctypes.c_int32),
                ("smem_per_cell_fp64", ctypes.c_int32), ("factor_updates", ctypes.c_int64),
                ("flops_forcing", ctypes.c_int64), ("flops_jacobian", ctypes.c_int64),
                ("flops_factor", ctypes.c_int64), ("flops_solve", ctypes.c_int64),
                ("env_rh", ctypes.c_int32), ("n_electrolytes", ctypes.c_int32),
                ("model_forcing", ctypes.c_int64), ("block_arrow", ctypes.c_int32),
                ("lanes_per_cell", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SolveOpts(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("max_steps", ctypes.c_int32), ("cells_per_block", ctypes.c_int32),
                ("hmin_frac", ctypes.c_double), ("stats", ctypes.c_void_p),
                ("workspace", ctypes.c_void_p), ("step", ctypes.c_void_p)]


class Group(ctypes.Structure):
    _fields_ = [("mech", ctypes.c_void_p), ("n_cells", ctypes.c_int64), ("state", ctypes.c_void_p),
                ("env", ctypes.c_void_p), ("atol", ctypes.c_void_p), ("atol_len", ctypes.c_int32),
                ("status", ctypes.c_void_p), ("stats", ctypes.c_void_p), ("workspace", ctypes.c_void_p),
                ("step", ctypes.c_void_p)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int32)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("n_cells", ctypes.c_int64), ("rc", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


E_TIMEOUT = -7
E_CANCELLED = -8
E_UNSUPPORTED = -5
E_BUDGET = -6

EXPORTS = ["camp_mech_load", "camp_mech_compile", "camp_mech_free", "camp_mech_info_get", "camp_mech_species_index",
           "camp_mech_structure", "camp_solve_opts_default", "camp_workspace_bytes", "camp_solve",
           "camp_solve_host", "camp_rate_constants", "camp_forcing", "camp_jacobian",
           "camp_lu_solve", "camp_last_error", "camp_server_create", "camp_server_submit",
           "camp_server_poll", "camp_server_wait", "camp_server_stats", "camp_server_cancel",
           "camp_server_destroy",
           "camp_solve_batch", "camp_solve_batch_host", "camp_autotune", "camp_mech_set_lanes", "camp_probe_fma_rate",
           "camp_solve_host_static", "camp_solve_sequence", "camp_server_resident_create", "camp_server_resident_step",
           "camp_server_resident_read", "camp_server_resident_write", "camp_server_resident_destroy"]


def lib():
    """Load libcamp.so (raises CampError if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise CampError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    L.camp_mech_load.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(vp),
                                 ctypes.c_char_p, ctypes.c_size_t]
    L.camp_mech_load.restype = ctypes.c_int
    L.camp_mech_compile.argtypes = L.camp_mech_load.argtypes
    L.camp_mech_compile.restype = ctypes.c_int
    L.camp_mech_free.argtypes = [vp]
    L.camp_mech_free.restype = None
    L.camp_mech_info_get.argtypes = [vp, ctypes.POINTER(MechInfo)]
    L.camp_mech_species_index.argtypes = [vp, ctypes.c_char_p]
    L.camp_mech_structure.argtypes = [vp] + [vp] * 8
    L.camp_solve_opts_default.argtypes = [ctypes.POINTER(SolveOpts), ctypes.c_int]
    L.camp_solve_opts_default.restype = None
    L.camp_workspace_bytes.restype = ctypes.c_size_t
    L.camp_solve.argtypes = [vp, i64, vp, vp, dbl, dbl, vp, i32, vp, ctypes.POINTER(SolveOpts), vp]
    L.camp_solve_host.argtypes = L.camp_solve.argtypes
    L.camp_solve_sequence.argtypes = [vp, i64, vp, vp, dbl, i32, vp, dbl, vp, i32, vp, ctypes.POINTER(SolveOpts), vp]
    L.camp_rate_constants.argtypes = [vp, i64, vp, vp, vp, vp]
    L.camp_forcing.argtypes = [vp, i64, vp, vp, vp, vp]
    L.camp_jacobian.argtypes = [vp, i64, vp, vp, vp, i32, vp]
    L.camp_lu_solve.argtypes = [vp, i64, vp, vp, dbl, vp, vp, vp, i32, vp]
    L.camp_last_error.restype = ctypes.c_char_p
    L.camp_server_create.argtypes = [ctypes.POINTER(ServerOpts), ctypes.POINTER(vp)]
    L.camp_server_submit.argtypes = [vp, vp, i64, vp, vp, dbl, dbl, dbl, vp, ctypes.POINTER(SolveOpts),
                                     ctypes.POINTER(ctypes.c_uint64)]
    L.camp_server_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(i32), ctypes.POINTER(RequestInfo)]
    L.camp_server_wait.argtypes = [vp, ctypes.c_uint64, i32, ctypes.POINTER(RequestInfo)]
    L.camp_server_stats.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_size_t)]
    L.camp_server_cancel.argtypes = [vp, ctypes.c_uint64]
    L.camp_server_destroy.argtypes = [vp]
    L.camp_server_resident_create.argtypes = [vp, vp, i64, vp, i32, ctypes.POINTER(vp)]
    L.camp_server_resident_step.argtypes = [vp, vp, vp, dbl, dbl, dbl, vp, ctypes.POINTER(SolveOpts),
                                            ctypes.POINTER(ctypes.c_uint64)]
    L.camp_server_resident_read.argtypes = [vp, vp, vp, vp, vp, i32]
    L.camp_server_resident_write.argtypes = [vp, vp, vp, i32]
    L.camp_server_resident_destroy.argtypes = [vp, vp]
    L.camp_solve_batch.argtypes = [ctypes.POINTER(Group), i32, dbl, dbl, ctypes.POINTER(SolveOpts), vp]
    L.camp_solve_batch_host.argtypes = L.camp_solve_batch.argtypes
    L.camp_mech_set_lanes.argtypes = [vp, i32]
    L.camp_autotune.argtypes = [vp, i64, vp, vp, dbl, dbl, vp, i32, i32, ctypes.POINTER(i32),
                                ctypes.POINTER(i32), ctypes.POINTER(dbl), vp]
    L.camp_probe_fma_rate.argtypes = [i32, ctypes.POINTER(dbl), vp]
    L.camp_solve_host_static.argtypes = L.camp_solve.argtypes
    _lib = L
    return L


def _check(rc):
    if rc != 0:
        raise CampError(f"camp error {rc}: {lib().camp_last_error().decode()}")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_f64(t, shape, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise CampError(f"{name} must be a contiguous float64 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise CampError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


class Mechanism:
    """A compiled mechanism whose tables live on the current CUDA device
    (device=False: compiled on the host only, for info and structure)."""

    def __init__(self, json_text: str, device: bool = True):
        L = lib()
        b = json_text.encode() if isinstance(json_text, str) else json_text
        h = ctypes.c_void_p()
        err = ctypes.create_string_buffer(1024)
        load = L.camp_mech_load if device else L.camp_mech_compile
        rc = load(b, len(b), ctypes.byref(h), err, len(err))
        if rc != 0:
            raise CampError(f"mechanism load failed ({rc}): {err.value.decode()}")
        self._h = h
        self.info = MechInfo()
        _check(L.camp_mech_info_get(self._h, ctypes.byref(self.info)))
        self.n = self.info.n_species
        self.n_env = self.info.n_env
        self.n_rxn = self.info.n_rxn

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.camp_mech_free(self._h)
            self._h = None

    def species_index(self, name):
        return lib().camp_mech_species_index(self._h, name.encode())

    def structure(self):
        inf = self.info
        n = self.n
        arrs = {"rowptr": n + 1, "colidx": inf.nnz_jac, "rxn_map": inf.rxn_map_len, "perm": n,
                "lu_rowptr": n + 1, "lu_colidx": inf.nnz_lu, "level_fwd": n, "level_bwd": n}
        out = {k: np.zeros(v, dtype=np.int32) for k, v in arrs.items()}
        _check(lib().camp_mech_structure(self._h, *[ctypes.c_void_p(out[k].ctypes.data) for k in arrs]))
        return out

    def _atol(self, atol, device):
        import torch
        a = torch.as_tensor(np.atleast_1d(np.asarray(atol, dtype=np.float64)), device=device)
        if a.numel() not in (1, self.n):
            raise CampError("atol must be a scalar or one value per species")
        return a.contiguous()

    def solve(self, state, env, dt, rtol, atol, status=None, variant=VARIANT_MIXED,
              persistent=None, max_steps=10000, cells_per_block=0, stats=None, workspace=None,
              stream=None, step=None):
        """Integrate every cell over [0, dt] in place (asynchronous on `stream`).

        state [C, n] / env [C, n_env]: float64 CUDA tensors; status: int32
        CUDA tensor [C] (allocated if None); stats: optional int32 [C, NSTATS];
        step: optional float64 CUDA tensor [C], in/out warm-start step sizes
        (camp_solve_opts.step).  Returns status.
        """
        import torch
        C = state.shape[0]
        _dev_f64(state, (C, self.n), "state")
        _dev_f64(env, (C, self.n_env), "env")
        if status is None:
            status = torch.empty(C, dtype=torch.int32, device=state.device)
        a = atol if isinstance(atol, torch.Tensor) else self._atol(atol, state.device)
        o = self.opts(variant, persistent, max_steps, cells_per_block, stats, workspace)
        if step is not None:
            _dev_f64(step, (C,), "step")
            o.step = step.data_ptr()
        _check(lib().camp_solve(self._h, C, _ptr(state), _ptr(env), float(dt), float(rtol), _ptr(a),
                                a.numel(), _ptr(status), ctypes.byref(o), _stream(stream)))
        return status

    def solve_sequence(self, state, env, dt, n_steps, rtol, atol, trajectory=None, status=None,
                       variant=VARIANT_MIXED, persistent=None, stats=None, stream=None, step=None,
                       max_steps=10000):
        """n_steps consecutive outer steps of dt in one launch (camp_solve_
        sequence); trajectory: optional float64 CUDA tensor [n_steps, C, n]
        receiving the state after every step.  Returns status."""
        import torch
        C = state.shape[0]
        _dev_f64(state, (C, self.n), "state")
        _dev_f64(env, (C, self.n_env), "env")
        if trajectory is not None:
            _dev_f64(trajectory, (n_steps, C, self.n), "trajectory")
        if status is None:
            status = torch.empty(C, dtype=torch.int32, device=state.device)
        a = atol if isinstance(atol, torch.Tensor) else self._atol(atol, state.device)
        o = self.opts(variant, persistent, max_steps=max_steps, stats=stats)
        if step is not None:
            _dev_f64(step, (C,), "step")
            o.step = step.data_ptr()
        _check(lib().camp_solve_sequence(self._h, C, _ptr(state), _ptr(env), float(dt), int(n_steps),
                                         _ptr(trajectory), float(rtol), _ptr(a), a.numel(), _ptr(status),
                                         ctypes.byref(o), _stream(stream)))
        return status

    def autotune(self, state, env, dt, rtol, atol, variant=VARIANT_MIXED, stream=None):
        """Pick cells-per-block and grid mapping by timing them on these cells
        (device tensors, left unchanged); returns (cpb, persistent, ms).  For
        129-256 species it also picks the cell shape (info.lanes_per_cell)."""
        C = state.shape[0]
        a = atol if hasattr(atol, "data_ptr") else self._atol(atol, state.device)
        cpb, pers, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        _check(lib().camp_autotune(self._h, C, _ptr(_dev_f64(state, (C, self.n), "state")),
                                   _ptr(_dev_f64(env, (C, self.n_env), "env")), float(dt), float(rtol),
                                   _ptr(a), a.numel(), variant, ctypes.byref(cpb), ctypes.byref(pers),
                                   ctypes.byref(ms), _stream(stream)))
        _check(lib().camp_mech_info_get(self._h, ctypes.byref(self.info)))
        return cpb.value, pers.value, ms.value

    def set_lanes(self, lanes):
        """Rebuild the per-lane tables for `lanes` threads a cell (the cell
        shape); refreshes info."""
        _check(lib().camp_mech_set_lanes(self._h, int(lanes)))
        _check(lib().camp_mech_info_get(self._h, ctypes.byref(self.info)))

    def opts(self, variant=VARIANT_MIXED, persistent=None, max_steps=10000, cells_per_block=0,
             stats=None, workspace=None):
        o = SolveOpts()
        lib().camp_solve_opts_default(ctypes.byref(o), variant)
        if persistent is not None:
            o.persistent = int(persistent)
        o.max_steps = max_steps
        o.cells_per_block = cells_per_block
        o.stats = stats.data_ptr() if stats is not None else None
        o.workspace = workspace.data_ptr() if workspace is not None else None
        return o

    def solve_host(self, state, env, dt, rtol, atol, variant=VARIANT_MIXED, persistent=None,
                   max_steps=10000, cells_per_block=0, stats=None, stream=None, step=None):
        """Host arrays (numpy float64, C-contiguous; pinned torch tensors also
        work): state is updated in place; returns the status array.  step:
        optional float64 array [C], in/out warm-start step sizes."""
        st = state if isinstance(state, np.ndarray) else state.numpy()
        ev = env if isinstance(env, np.ndarray) else env.numpy()
        if st.dtype != np.float64 or not st.flags.c_contiguous or st.shape[1] != self.n:
            raise CampError("state must be C-contiguous float64 [C, n]")
        if ev.dtype != np.float64 or not ev.flags.c_contiguous or ev.shape != (st.shape[0], self.n_env):
            raise CampError("env must be C-contiguous float64 [C, n_env]")
        a = np.ascontiguousarray(np.atleast_1d(np.asarray(atol, dtype=np.float64)))
        status = np.zeros(st.shape[0], dtype=np.int32)
        o = SolveOpts()
        lib().camp_solve_opts_default(ctypes.byref(o), variant)
        if persistent is not None:
            o.persistent = int(persistent)
        o.max_steps = max_steps
        o.cells_per_block = cells_per_block
        o.stats = stats.ctypes.data if stats is not None else None
        if step is not None:
            if step.dtype != np.float64 or not step.flags.c_contiguous or step.shape != (st.shape[0],):
                raise CampError("step must be C-contiguous float64 [C]")
            o.step = step.ctypes.data
        _check(lib().camp_solve_host(self._h, st.shape[0], ctypes.c_void_p(st.ctypes.data),
                                     ctypes.c_void_p(ev.ctypes.data), float(dt), float(rtol),
                                     ctypes.c_void_p(a.ctypes.data), a.size,
                                     ctypes.c_void_p(status.ctypes.data), ctypes.byref(o),
                                     _stream(stream)))
        return status

    # ---- single steps of the method (test entry points) ----
    def rate_constants(self, env, stream=None):
        import torch
        C = env.shape[0]
        _dev_f64(env, (C, self.n_env), "env")
        kf = torch.empty((C, self.n_rxn), dtype=torch.float64, device=env.device)
        kr = torch.empty_like(kf)
        _check(lib().camp_rate_constants(self._h, C, _ptr(env), _ptr(kf), _ptr(kr), _stream(stream)))
        return kf, kr

    def forcing(self, state, env, stream=None):
        import torch
        C = state.shape[0]
        f = torch.empty((C, self.n), dtype=torch.float64, device=state.device)
        _check(lib().camp_forcing(self._h, C, _ptr(_dev_f64(state, (C, self.n), "state")),
                                  _ptr(_dev_f64(env, (C, self.n_env), "env")), _ptr(f), _stream(stream)))
        return f

    def jacobian(self, state, env, variant=VARIANT_FP64, stream=None):
        import torch
        C = state.shape[0]
        J = torch.empty((C, self.info.nnz_jac), dtype=torch.float64, device=state.device)
        _check(lib().camp_jacobian(self._h, C, _ptr(_dev_f64(state, (C, self.n), "state")),
                                   _ptr(_dev_f64(env, (C, self.n_env), "env")), _ptr(J), variant,
                                   _stream(stream)))
        return J

    def lu_solve(self, state, env, gamma, b, variant=VARIANT_FP64, stream=None):
        import torch
        C = state.shape[0]
        x = torch.empty((C, self.n), dtype=torch.float64, device=state.device)
        st = torch.empty(C, dtype=torch.int32, device=state.device)
        _check(lib().camp_lu_solve(self._h, C, _ptr(_dev_f64(state, (C, self.n), "state")),
                                   _ptr(_dev_f64(env, (C, self.n_env), "env")), float(gamma),
                                   _ptr(_dev_f64(b, (C, self.n), "b")), _ptr(x), _ptr(st), variant,
                                   _stream(stream)))
        return x, st


class Server:
    """Continuous-batching request loop (camp_server_*): chunks of cells on
    host buffers, admitted under a device-memory budget, overlapped on the
    GPU.  Buffers passed to submit() must stay alive until the request
    finishes; pinned memory lets copies overlap."""

    def __init__(self, hbm_budget_bytes, max_inflight=8):
        o = ServerOpts(int(hbm_budget_bytes), int(max_inflight))
        h = ctypes.c_void_p()
        _check(lib().camp_server_create(ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, mech, state, env, dt, rtol, atol, status, variant=VARIANT_MIXED, persistent=None):
        """state/env: C-contiguous float64 host arrays (numpy or pinned torch);
        status: int32 host array.  Returns the request id."""
        st = state if isinstance(state, np.ndarray) else state.numpy()
        ev = env if isinstance(env, np.ndarray) else env.numpy()
        ss = status if isinstance(status, np.ndarray) else status.numpy()
        if st.shape[1] != mech.n or ev.shape != (st.shape[0], mech.n_env) or ss.shape != (st.shape[0],):
            raise CampError("shape mismatch")
        o = mech.opts(variant, persistent)
        rid = ctypes.c_uint64()
        _check(lib().camp_server_submit(self._h, mech._h, st.shape[0], ctypes.c_void_p(st.ctypes.data),
                                        ctypes.c_void_p(ev.ctypes.data), float(dt), float(rtol),
                                        float(atol), ctypes.c_void_p(ss.ctypes.data), ctypes.byref(o),
                                        ctypes.byref(rid)))
        self._keep[rid.value] = (state, env, status, mech)
        return rid.value

    def wait(self, rid, timeout_ms=600000):
        """Request info dict, or None on timeout (the request stays queued)."""
        info = RequestInfo()
        rc = lib().camp_server_wait(self._h, rid, int(timeout_ms), ctypes.byref(info))
        if rc == E_TIMEOUT:
            return None
        _check(rc)
        self._keep.pop(rid, None)
        return info.as_dict()

    def poll(self, rid):
        info = RequestInfo()
        done = ctypes.c_int32()
        _check(lib().camp_server_poll(self._h, rid, ctypes.byref(done), ctypes.byref(info)))
        if not done.value:
            return None
        self._keep.pop(rid, None)
        return info.as_dict()

    def cancel(self, rid):
        """Withdraw a request still waiting for admission: True if withdrawn
        (it then finishes with rc E_CANCELLED), False if already on the GPU
        or finished."""
        rc = lib().camp_server_cancel(self._h, rid)
        if rc == E_UNSUPPORTED:
            return False
        _check(rc)
        return True

    def resident(self, mech, state, warm_start=False):
        """A resident cell set initialised from the host array state [C, n]
        (copied in; the set keeps its state on the device)."""
        return Resident(self, mech, state, warm_start)

    def stats(self):
        p, i, b = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_size_t()
        _check(lib().camp_server_stats(self._h, ctypes.byref(p), ctypes.byref(i), ctypes.byref(b)))
        return {"pending": p.value, "inflight": i.value, "bytes_in_use": b.value}

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().camp_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        if _lib is not None:
            self.close()


class Resident:
    """A chunk whose state stays on the device across the host's steps
    (camp_server_resident_*).  step() queues one step (env copied in at
    admission; keep env alive until the request finishes); read() / write()
    move the state on demand."""

    def __init__(self, server, mech, state, warm_start=False):
        st = np.ascontiguousarray(state, dtype=np.float64)
        if st.ndim != 2 or st.shape[1] != mech.n:
            raise CampError("state must be [C, n_species]")
        h = ctypes.c_void_p()
        _check(lib().camp_server_resident_create(server._h, mech._h, st.shape[0], ctypes.c_void_p(st.ctypes.data),
                                                 int(bool(warm_start)), ctypes.byref(h)))
        self._srv, self._h, self.mech, self.n_cells = server, h, mech, st.shape[0]

    def step(self, env, dt, rtol, atol, status=None, variant=VARIANT_MIXED, persistent=None):
        ev = env if isinstance(env, np.ndarray) else env.numpy()
        if ev.dtype != np.float64 or not ev.flags.c_contiguous or ev.shape != (self.n_cells, self.mech.n_env):
            raise CampError("env must be C-contiguous float64 [C, n_env]")
        ss = None
        if status is not None:
            ss = status if isinstance(status, np.ndarray) else status.numpy()
            if ss.dtype != np.int32 or ss.shape != (self.n_cells,):
                raise CampError("status must be int32 [C]")
        o = self.mech.opts(variant, persistent)
        rid = ctypes.c_uint64()
        _check(lib().camp_server_resident_step(self._srv._h, self._h, ctypes.c_void_p(ev.ctypes.data), float(dt),
                                               float(rtol), float(atol),
                                               ctypes.c_void_p(ss.ctypes.data) if ss is not None else None,
                                               ctypes.byref(o), ctypes.byref(rid)))
        self._srv._keep[rid.value] = (env, status, self)
        return rid.value

    def read(self, timeout_ms=600000, with_step=False):
        """(state [C, n], status of the last step [C][, carried step sizes])"""
        y = np.zeros((self.n_cells, self.mech.n))
        st = np.zeros(self.n_cells, dtype=np.int32)
        hs = np.zeros(self.n_cells) if with_step else None
        _check(lib().camp_server_resident_read(self._srv._h, self._h, ctypes.c_void_p(y.ctypes.data),
                                               ctypes.c_void_p(st.ctypes.data),
                                               ctypes.c_void_p(hs.ctypes.data) if hs is not None else None,
                                               int(timeout_ms)))
        return (y, st, hs) if with_step else (y, st)

    def write(self, state, timeout_ms=600000):
        st = np.ascontiguousarray(state, dtype=np.float64)
        if st.shape != (self.n_cells, self.mech.n):
            raise CampError("state must be [C, n_species]")
        _check(lib().camp_server_resident_write(self._srv._h, self._h, ctypes.c_void_p(st.ctypes.data),
                                                int(timeout_ms)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._srv._h is not None:
            _check(lib().camp_server_resident_destroy(self._srv._h, self._h))
        self._h = None


def workspace(device):
    """Device scratch for one concurrent solve (the work counter)."""
    import torch
    return torch.zeros(int(lib().camp_workspace_bytes()), dtype=torch.uint8, device=device)


def solve_batch(groups, dt, rtol, variant=VARIANT_MIXED, stream=None):
    """groups: list of dicts {mech, state, env, atol (tensor), status, stats?,
    workspace?, step?} of device tensors; one call, one persistent grid per group."""
    arr = (Group * len(groups))()
    for i, g in enumerate(groups):
        m = g["mech"]
        C = g["state"].shape[0]
        _dev_f64(g["state"], (C, m.n), "state")
        _dev_f64(g["env"], (C, m.n_env), "env")
        arr[i] = Group(m._h.value, C, g["state"].data_ptr(), g["env"].data_ptr(), g["atol"].data_ptr(),
                       g["atol"].numel(), g["status"].data_ptr(),
                       g["stats"].data_ptr() if g.get("stats") is not None else None,
                       g["workspace"].data_ptr() if g.get("workspace") is not None else None,
                       g["step"].data_ptr() if g.get("step") is not None else None)
    o = SolveOpts()
    lib().camp_solve_opts_default(ctypes.byref(o), variant)
    _check(lib().camp_solve_batch(arr, len(groups), float(dt), float(rtol), ctypes.byref(o), _stream(stream)))


def _host_arr(a, dtype, shape, name):
    a = a if isinstance(a, np.ndarray) else a.numpy()
    if a.dtype != dtype or not a.flags.c_contiguous or tuple(a.shape) != tuple(shape):
        raise CampError(f"{name} must be a C-contiguous {np.dtype(dtype).name} host array of shape {shape}")
    return a


def solve_batch_host(groups, dt, rtol, variant=VARIANT_MIXED, stream=None):
    """groups: list of dicts {mech, state, env, atol, status, stats?, step?}
    of host arrays (numpy, or pinned torch tensors); states are updated in
    place.  One synchronous call: copies in, one camp_solve_batch, copies out."""
    arr = (Group * len(groups))()
    keep = []
    for i, g in enumerate(groups):
        m = g["mech"]
        st = g["state"] if isinstance(g["state"], np.ndarray) else g["state"].numpy()
        C = st.shape[0]
        st = _host_arr(st, np.float64, (C, m.n), "state")
        ev = _host_arr(g["env"], np.float64, (C, m.n_env), "env")
        a = np.ascontiguousarray(np.atleast_1d(np.asarray(g["atol"], dtype=np.float64)))
        ss = _host_arr(g["status"], np.int32, (C,), "status")
        stats = _host_arr(g["stats"], np.int32, (C, NSTATS), "stats") if g.get("stats") is not None else None
        step = _host_arr(g["step"], np.float64, (C,), "step") if g.get("step") is not None else None
        keep += [st, ev, a, ss, stats, step]
        arr[i] = Group(m._h.value, C, st.ctypes.data, ev.ctypes.data, a.ctypes.data, a.size, ss.ctypes.data,
                       stats.ctypes.data if stats is not None else None, None,
                       step.ctypes.data if step is not None else None)
    o = SolveOpts()
    lib().camp_solve_opts_default(ctypes.byref(o), variant)
    _check(lib().camp_solve_batch_host(arr, len(groups), float(dt), float(rtol), ctypes.byref(o),
                                       _stream(stream)))


def probe_fma_rate(fp64=True, stream=None):
    """Measured FMA throughput of the current GPU, GFLOP/s."""
    g = ctypes.c_double()
    _check(lib().camp_probe_fma_rate(int(fp64), ctypes.byref(g), _stream(stream)))
    return g.value
