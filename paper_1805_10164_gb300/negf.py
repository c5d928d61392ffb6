"""Thin ctypes binding of libnegf (include/negf.h).  Argument marshalling only: every step of
the walk path runs in the library's CUDA kernels.  Functions carry the C entry points' names.

Device memory and streams come from PyTorch: a context binds ``torch.cuda.current_stream()``
unless a stream is given, and device-resident wire arrays may be torch CUDA tensors.
The library must have been built (``paper_1805_10164_gb300.build.build()``); loading fails
loudly otherwise - there is no fallback.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

NEGF_OK, NEGF_E_INVALID, NEGF_E_NOMEM, NEGF_E_CUDA, NEGF_E_NUMERIC, NEGF_E_STEPCAP, NEGF_E_TIMEOUT = range(7)
PRECISION = {"fp64": 0, "fp32": 1, "split_tf32": 2}
EXPORT = {"alias": 0, "mode_alias": 1, "weights": 2, "mode_weights": 3, "rowsum": 4,
          "alias_level1": 5}
LAYOUT = {"auto": 0, "one_level": 1, "two_level": 2}
TALLY_FIELDS = 5
MAX_STEPS = 1 << 24
_STATUS = {0: "NEGF_OK", 1: "NEGF_E_INVALID", 2: "NEGF_E_NOMEM", 3: "NEGF_E_CUDA",
           4: "NEGF_E_NUMERIC", 5: "NEGF_E_STEPCAP", 6: "NEGF_E_TIMEOUT"}


class NegfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class negf_wire(C.Structure):
    _fields_ = [("W", C.c_int32), ("L", C.c_int32), ("t", C.c_double),
                ("onsite", C.c_void_p), ("eta", C.c_void_p), ("n_energy", C.c_int32),
                ("energy", C.c_void_p), ("energy_weight", C.c_void_p),
                ("lead_model", C.c_int32), ("gamma_lead", C.c_double),
                ("slice_h", C.c_void_p)]


class negf_build_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("memspace", C.c_int32), ("keep_weights", C.c_int32),
                ("keep_green", C.c_int32), ("table_layout", C.c_int32)]


class negf_task_info(C.Structure):
    _fields_ = [("wire", C.c_int32), ("energy_index", C.c_int32), ("W", C.c_int32),
                ("L", C.c_int32), ("n", C.c_int32), ("K", C.c_int32), ("rows", C.c_int32),
                ("table_layout", C.c_int32), ("energy", C.c_double), ("energy_weight", C.c_double),
                ("c", C.c_double * 2), ("table_offset", C.c_uint64), ("mode_offset", C.c_uint64)]


class negf_run_opts(C.Structure):
    _fields_ = [("start_lead", C.c_int32), ("tasks_per_wave", C.c_int32), ("seed", C.c_uint64),
                ("walkers_per_task", C.c_uint64), ("walker_id_offset", C.c_uint64),
                ("max_steps", C.c_uint32), ("waves_in_flight", C.c_int32),
                ("memory_budget", C.c_uint64), ("walk_blocks_per_sm", C.c_int32),
                ("reserved", C.c_int32)]


_lib = None


class negf_plan_tuning(C.Structure):
    _fields_ = [("walk_blocks_per_sm", C.c_int32), ("chain_warps", C.c_int32),
                ("alias_warps", C.c_int32), ("tuned", C.c_int32), ("walk_ms", C.c_float),
                ("chain_ms", C.c_float), ("alias_ms", C.c_float), ("walk_slots", C.c_int32)]


class negf_thermal_result(C.Structure):
    _fields_ = [("G", C.c_double), ("se", C.c_double), ("window", C.c_double),
                ("mean_steps", C.c_double), ("walkers", C.c_uint64),
                ("absorbed", C.c_uint64 * 2), ("closed", C.c_uint64), ("truncated", C.c_uint64)]


def library_path():
    return _build.LIB


def load():
    """Load libnegf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libnegf.so is not built ({path}); call "
                           "paper_1805_10164_gb300.build.build() first")
    lib = C.CDLL(path)
    P, I32, U32, U64, D = C.c_void_p, C.c_int32, C.c_uint32, C.c_uint64, C.c_double
    sig = {
        "negf_abi_version": (C.c_int, []),
        "negf_device_error_status": (I32, [I32, C.c_char_p, C.c_size_t]),
        "negf_create": (I32, [C.POINTER(P), C.c_int, P]),
        "negf_destroy": (None, [P]),
        "negf_last_error": (C.c_char_p, [P]),
        "negf_build_tables": (I32, [P, C.POINTER(negf_wire), I32, C.POINTER(negf_build_opts),
                                    C.POINTER(P)]),
        "negf_tables_num_tasks": (I32, [P]),
        "negf_tables_num_wires": (I32, [P]),
        "negf_tables_device_bytes": (U64, [P]),
        "negf_get_task_info": (I32, [P, P, I32, C.POINTER(negf_task_info)]),
        "negf_tables_free": (None, [P]),
        "negf_export_tables": (I32, [P, P, I32, I32, P, C.POINTER(C.c_size_t)]),
        "negf_export_table_rows": (I32, [P, P, I32, I32, C.c_int64, C.c_int64, P,
                                         C.POINTER(C.c_size_t)]),
        "negf_walk": (I32, [P, P, I32, U64, U64, U64, U32, C.POINTER(P)]),
        "negf_walk_trace": (I32, [P, P, I32, I32, U64, U64, U64, U32, P, P]),
        "negf_tally_counts": (I32, [P, P, P]),
        "negf_tally_accumulate": (I32, [P, P, P]),
        "negf_tally_start_lead": (I32, [P]),
        "negf_tally_free": (None, [P]),
        "negf_current": (I32, [P, P, P, D, D, D, P, P, P, P]),
        "negf_profile_enable": (I32, [P, I32]),
        "negf_build_tables_noalloc": (I32, [C.POINTER(negf_wire), I32, P, P, P, P]),
        "negf_run": (I32, [P, C.POINTER(negf_wire), I32, C.POINTER(negf_build_opts),
                           C.POINTER(negf_run_opts), C.POINTER(P), C.POINTER(P)]),
        "negf_tables_num_waves": (I32, [P]),
        "negf_probe_gather": (I32, [P, U64, I32, I32, C.POINTER(D)]),
        "negf_walk_score": (I32, [P, P, I32, U64, U64, U64, U32, C.POINTER(P)]),
        "negf_walk_inelastic": (I32, [P, P, I32, U64, U64, U64, U32, C.c_double, C.POINTER(P)]),
        "negf_export_energy_tables": (I32, [P, P, I32, C.c_double, P, C.POINTER(C.c_size_t)]),
        "negf_tally_score_counts": (I32, [P, P, P, P]),
        "negf_tally_score_accumulate": (I32, [P, P, P, P]),
        "negf_tally_score_size": (U64, [P]),
        "negf_tally_mode_size": (U32, [P]),
        "negf_current_backward": (I32, [P, P, P, D, D, D, P, P, P]),
        "negf_current_backward_rgf": (I32, [P, P, P, D, D, D, P, I32, P, P]),
        "negf_plan_create": (I32, [P, C.POINTER(negf_wire), I32, C.POINTER(negf_build_opts),
                                   C.POINTER(negf_run_opts), D, D, D, I32, C.POINTER(P)]),
        "negf_plan_launch": (I32, [P, P, U64, U64]),
        "negf_plan_result": (I32, [P, P, P, P, P, P, P]),
        "negf_plan_get_tuning": (I32, [P, C.POINTER(negf_plan_tuning)]),
        "negf_plan_num_tasks": (I32, [P]),
        "negf_plan_num_waves": (I32, [P]),
        "negf_plan_device_bytes": (U64, [P]),
        "negf_plan_destroy": (None, [P]),
        "negf_profile_read": (I32, [P, I32, P, P, P, C.POINTER(I32)]),
        "negf_walk_thermal": (I32, [P, P, I32, I32, U64, U64, U64, D, D, U32, P, P, P, P,
                                    C.POINTER(negf_thermal_result)]),
        "negf_interval_distance": (I32, [P, P, I32, I32, P]),
        "negf_thermal_grid": (I32, [P, C.POINTER(negf_wire), I32, D, D, I32, D, I32, I32, P,
                                    C.POINTER(I32)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(ctx, st, allow=()):
    if st != NEGF_OK and st not in allow:
        msg = load().negf_last_error(ctx)
        raise NegfError(st, msg.decode() if msg else "")
    return st


def _ptr(x):
    """Address of a numpy array (host) or torch tensor (device/host)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def negf_create(device=0, stream=None):
    import torch
    lib = load()
    if stream is None:
        stream = torch.cuda.current_stream(device)
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    out = C.c_void_p()
    st = lib.negf_create(C.byref(out), int(device), C.c_void_p(handle))
    if st != NEGF_OK:
        raise NegfError(st, "negf_create failed")
    return out


def negf_destroy(ctx):
    load().negf_destroy(ctx)


def _wire_array(wires, memspace, keep):
    arr = (negf_wire * max(1, len(wires)))()
    for i, w in enumerate(wires):
        sh = getattr(w, "slice_h", None)
        if memspace == "host":
            on = np.ascontiguousarray(w.onsite, dtype=np.float64).reshape(-1)
            et = np.ascontiguousarray(w.eta, dtype=np.float64).reshape(-1)
            E = np.ascontiguousarray(w.energy, dtype=np.float64).reshape(-1)
            wE = None if w.energy_weight is None else np.ascontiguousarray(
                w.energy_weight, dtype=np.float64).reshape(-1)
            sh = None if sh is None else np.ascontiguousarray(sh, dtype=np.float64).reshape(-1)
        else:
            on, et, E, wE, sh = (t.contiguous() if t is not None else None
                                 for t in (w.onsite, w.eta, w.energy, w.energy_weight, sh))
        keep.extend([on, et, E, wE, sh])
        arr[i] = negf_wire(int(w.W), int(w.L), float(w.t), _ptr(on), _ptr(et), int(len(E)),
                           _ptr(E), _ptr(wE), int(getattr(w, "lead_model", 0)),
                           float(getattr(w, "gamma_lead", 0.0)), _ptr(sh))
    return arr


def negf_run(ctx, wires, start_lead, seed, walkers_per_task, precision="fp32", memspace="host",
             walker_id_offset=0, max_steps=1 << 20, tasks_per_wave=0, waves_in_flight=0,
             memory_budget=0, walk_blocks_per_sm=0, layout="auto"):
    """Build + walk pipelined in waves.  Returns (tasks handle, tally handle)."""
    lib = load()
    keep = []
    arr = _wire_array(wires, memspace, keep)
    bopts = negf_build_opts(PRECISION[precision], 0 if memspace == "host" else 1, 0, 0,
                            LAYOUT[layout])
    ropts = negf_run_opts(int(start_lead), int(tasks_per_wave), int(seed), int(walkers_per_task),
                          int(walker_id_offset), int(max_steps), int(waves_in_flight),
                          int(memory_budget), int(walk_blocks_per_sm), 0)
    t_out, tl_out = C.c_void_p(), C.c_void_p()
    _check(ctx, lib.negf_run(ctx, arr, len(wires), C.byref(bopts), C.byref(ropts),
                             C.byref(t_out), C.byref(tl_out)))
    del keep
    return t_out, tl_out


def negf_tables_num_waves(tables):
    return load().negf_tables_num_waves(tables)


def negf_build_tables(ctx, wires, precision="fp64", memspace="host", keep_weights=False,
                      keep_green=False, layout="auto"):
    """wires: objects with W, L, t, onsite, eta, energy, energy_weight, lead_model, gamma_lead
    (numpy float64 arrays for memspace 'host', torch CUDA float64 tensors for 'device')."""
    lib = load()
    keep = []
    arr = _wire_array(wires, memspace, keep)
    opts = negf_build_opts(PRECISION[precision], 0 if memspace == "host" else 1,
                           1 if keep_weights else 0, 1 if keep_green else 0, LAYOUT[layout])
    out = C.c_void_p()
    _check(ctx, lib.negf_build_tables(ctx, arr, len(wires), C.byref(opts), C.byref(out)))
    del keep
    return out


def negf_tables_num_tasks(tables):
    return load().negf_tables_num_tasks(tables)


def negf_tables_device_bytes(tables):
    return load().negf_tables_device_bytes(tables)


def negf_get_task_info(ctx, tables, task):
    info = negf_task_info()
    _check(ctx, load().negf_get_task_info(ctx, tables, int(task), C.byref(info)))
    return dict(wire=info.wire, energy_index=info.energy_index, W=info.W, L=info.L, n=info.n,
                K=info.K, rows=info.rows, energy=info.energy, energy_weight=info.energy_weight,
                c=np.array([info.c[0], info.c[1]]), table_offset=info.table_offset,
                layout={1: "one_level", 2: "two_level"}.get(info.table_layout, "unknown"),
                mode_offset=info.mode_offset)


def negf_tables_free(tables):
    load().negf_tables_free(tables)


def level2_words(W):
    """u32 words of one level-2 block of a two-level table (NEGF_LEVEL2_WORDS)."""
    return 8 if W <= 8 else 8 + 8 * ((W + 7) // 8)


def negf_export_tables(ctx, tables, task, what):
    lib = load()
    kind = EXPORT[what]
    nbytes = C.c_size_t(0)
    _check(ctx, lib.negf_export_tables(ctx, tables, int(task), kind, None, C.byref(nbytes)))
    dtype = np.uint64 if what in ("alias", "mode_alias", "alias_level1") else np.float64
    buf = np.empty(nbytes.value // 8, dtype=dtype)
    _check(ctx, lib.negf_export_tables(ctx, tables, int(task), kind, buf.ctypes.data,
                                       C.byref(nbytes)))
    return buf


def negf_export_table_rows(ctx, tables, task, what, row0, n_rows):
    """Rows [row0, row0 + n_rows) of one task's alias / alias_level1 (uint64) or rowsum
    (float64) data (the level-2 blocks of a two-level task: view the result as uint32)."""
    lib = load()
    kind = EXPORT[what]
    nbytes = C.c_size_t(0)
    _check(ctx, lib.negf_export_table_rows(ctx, tables, int(task), kind, int(row0), int(n_rows),
                                           None, C.byref(nbytes)))
    buf = np.empty(nbytes.value // 8, dtype=np.float64 if what == "rowsum" else np.uint64)
    _check(ctx, lib.negf_export_table_rows(ctx, tables, int(task), kind, int(row0), int(n_rows),
                                           buf.ctypes.data, C.byref(nbytes)))
    return buf


def negf_walk(ctx, tables, start_lead, seed, walkers_per_task, walker_id_offset=0,
              max_steps=1 << 20):
    out = C.c_void_p()
    _check(ctx, load().negf_walk(ctx, tables, int(start_lead), int(seed), int(walkers_per_task),
                                 int(walker_id_offset), int(max_steps), C.byref(out)))
    return out


def negf_walk_trace(ctx, tables, task, start_lead, seed, walker_id_offset, d_lead, d_steps,
                    max_steps=1 << 20):
    """d_lead: torch int32 CUDA tensor, d_steps: torch int32/uint32 CUDA tensor (n_walkers)."""
    n = int(d_lead.numel())
    _check(ctx, load().negf_walk_trace(ctx, tables, int(task), int(start_lead), int(seed),
                                       int(walker_id_offset), n, int(max_steps), _ptr(d_lead),
                                       _ptr(d_steps)))


def negf_walk_thermal(ctx, tables, wire, start_lead, seed, walkers, mu, kT,
                      walker_id_offset=0, max_steps=1 << 20, trace=None):
    """Linear conductance G_qp (units e^2/h) with energies drawn from the thermal window and
    transition probabilities interpolated on wire ``wire``'s energy grid.  trace: optional dict
    of torch CUDA tensors 'lead' (int32), 'steps' (int32), 'interval' (int32), 'a' (int32,
    read as uint32) of ``walkers`` entries each."""
    out = negf_thermal_result()
    tr = trace or {}
    st = load().negf_walk_thermal(ctx, tables, int(wire), int(start_lead), int(seed),
                                  int(walkers), int(walker_id_offset), float(mu), float(kT),
                                  int(max_steps), _ptr(tr.get("lead")), _ptr(tr.get("steps")),
                                  _ptr(tr.get("interval")), _ptr(tr.get("a")), C.byref(out))
    _check(ctx, st, allow=(NEGF_E_STEPCAP,))
    return dict(G=out.G, se=out.se, window=out.window, mean_steps=out.mean_steps,
                walkers=out.walkers, absorbed=(out.absorbed[0], out.absorbed[1]),
                closed=out.closed, truncated=out.truncated, stepcap=st == NEGF_E_STEPCAP)


def negf_tally_counts(ctx, tally, n_tasks):
    buf = np.zeros((n_tasks, TALLY_FIELDS), dtype=np.uint64)
    _check(ctx, load().negf_tally_counts(ctx, tally, buf.ctypes.data))
    return buf


def negf_tally_accumulate(ctx, tally, counts):
    counts = np.ascontiguousarray(counts, dtype=np.uint64)
    _check(ctx, load().negf_tally_accumulate(ctx, tally, counts.ctypes.data))


def negf_tally_free(tally):
    load().negf_tally_free(tally)


def negf_current(ctx, tables, tally, mu_p, mu_q, kT):
    """Returns dict(I, se, T, T_se, stepcap) with I/se per wire and T/T_se per task."""
    lib = load()
    nw = lib.negf_tables_num_wires(tables)
    nt = lib.negf_tables_num_tasks(tables)
    I = np.zeros(max(nw, 1))
    se = np.zeros(max(nw, 1))
    T = np.zeros(max(nt, 1))
    Tse = np.zeros(max(nt, 1))
    st = _check(ctx, lib.negf_current(ctx, tables, tally, float(mu_p), float(mu_q), float(kT),
                                      I.ctypes.data, se.ctypes.data, T.ctypes.data,
                                      Tse.ctypes.data), allow=(NEGF_E_STEPCAP,))
    return dict(I=I[:nw], se=se[:nw], T=T[:nt], T_se=Tse[:nt], stepcap=st == NEGF_E_STEPCAP)


def negf_profile_enable(ctx, on=True):
    _check(ctx, load().negf_profile_enable(ctx, 1 if on else 0))


def negf_profile_read(ctx, cap=32):
    """{kernel name: (launch groups, total device ms)} accumulated since profiling was enabled."""
    names = C.create_string_buffer(32 * cap)
    launches = np.zeros(cap, dtype=np.uint64)
    ms = np.zeros(cap)
    n = C.c_int32(0)
    _check(ctx, load().negf_profile_read(ctx, cap, names, launches.ctypes.data, ms.ctypes.data,
                                         C.byref(n)))
    out = {}
    raw = names.raw
    for i in range(min(n.value, cap)):
        name = raw[32 * i:32 * (i + 1)].split(b"\0", 1)[0].decode()
        out[name] = (int(launches[i]), float(ms[i]))
    return out


def negf_build_tables_noalloc(wire, precision, stream, d_alias, d_mode_alias, d_c):
    """Table build of one wire (host arrays) into caller-owned torch CUDA buffers, with all
    scratch in the library's fixed device array (no allocation).  Returns the status code."""
    on = np.ascontiguousarray(wire.onsite, dtype=np.float64).reshape(-1)
    et = np.ascontiguousarray(wire.eta, dtype=np.float64).reshape(-1)
    E = np.ascontiguousarray(wire.energy, dtype=np.float64).reshape(-1)
    sh = getattr(wire, "slice_h", None)
    sh = None if sh is None else np.ascontiguousarray(sh, dtype=np.float64).reshape(-1)
    w = negf_wire(int(wire.W), int(wire.L), float(wire.t), _ptr(on), _ptr(et), int(len(E)),
                  _ptr(E), None, int(getattr(wire, "lead_model", 0)),
                  float(getattr(wire, "gamma_lead", 0.0)), _ptr(sh))
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    return load().negf_build_tables_noalloc(C.byref(w), PRECISION[precision], C.c_void_p(handle),
                                            _ptr(d_alias), _ptr(d_mode_alias), _ptr(d_c))


def negf_interval_distance(ctx, tables, wire, n_energy, start_lead=0):
    """Distances of the wire's consecutive energies' Step 6' probabilities (n_energy - 1)."""
    d = np.zeros(max(n_energy - 1, 1))
    _check(ctx, load().negf_interval_distance(ctx, tables, int(wire), int(start_lead),
                                              d.ctypes.data))
    return d[:n_energy - 1]


def negf_thermal_grid(ctx, wire, e_lo, e_hi, n_init, tol=0.05, max_points=257,
                      precision="fp64", start_lead=0):
    """The interpolating sampler's grid on [e_lo, e_hi] (ascending energies)."""
    keep = []
    arr = _wire_array([wire], "host", keep)
    out = np.zeros(int(max_points))
    n = C.c_int32(0)
    _check(ctx, load().negf_thermal_grid(ctx, arr, PRECISION[precision], float(e_lo),
                                         float(e_hi), int(n_init), float(tol), int(max_points),
                                         int(start_lead), out.ctypes.data, C.byref(n)))
    return out[:n.value].copy()


def negf_device_error_status(word):
    """(status, description) a device error word is reported as (host only)."""
    buf = C.create_string_buffer(256)
    st = load().negf_device_error_status(int(word), buf, len(buf))
    return st, buf.value.decode()


def negf_probe_gather(ctx, table_bytes, ilp=8, chain=64):
    """Achieved random 8-byte gathers per second over a device table of table_bytes."""
    out = C.c_double(0.0)
    _check(ctx, load().negf_probe_gather(ctx, int(table_bytes), int(ilp), int(chain),
                                         C.byref(out)))
    return out.value


def negf_walk_inelastic(ctx, tables, start_lead, seed, walkers_per_task, sigma_E,
                        walker_id_offset=0, max_steps=1 << 20):
    out = C.c_void_p()
    _check(ctx, load().negf_walk_inelastic(ctx, tables, int(start_lead), int(seed),
                                           int(walkers_per_task), int(walker_id_offset),
                                           int(max_steps), float(sigma_E), C.byref(out)))
    return out


def negf_export_energy_tables(ctx, tables, task, sigma_E):
    """The Step 7' energy rows of a task: uint64 [n, nE] alias entries."""
    lib = load()
    nbytes = C.c_size_t(0)
    _check(ctx, lib.negf_export_energy_tables(ctx, tables, int(task), float(sigma_E), None,
                                              C.byref(nbytes)))
    buf = np.empty(nbytes.value // 8, dtype=np.uint64)
    _check(ctx, lib.negf_export_energy_tables(ctx, tables, int(task), float(sigma_E),
                                              buf.ctypes.data, C.byref(nbytes)))
    info = negf_get_task_info(ctx, tables, task)
    return buf.reshape(info["n"], -1)


def negf_walk_score(ctx, tables, start_lead, seed, walkers_per_task, walker_id_offset=0,
                    max_steps=1 << 20):
    out = C.c_void_p()
    _check(ctx, load().negf_walk_score(ctx, tables, int(start_lead), int(seed),
                                       int(walkers_per_task), int(walker_id_offset),
                                       int(max_steps), C.byref(out)))
    return out


def negf_tally_score_counts(ctx, tally):
    lib = load()
    ns, nm = lib.negf_tally_score_size(tally), lib.negf_tally_mode_size(tally)
    c = np.zeros((2, ns), dtype=np.uint64)
    m = np.zeros((2, nm), dtype=np.uint64)
    _check(ctx, lib.negf_tally_score_counts(ctx, tally, c.ctypes.data, m.ctypes.data))
    return c, m


def negf_tally_score_accumulate(ctx, tally, counts, mode_counts):
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    m = np.ascontiguousarray(mode_counts, dtype=np.uint64)
    _check(ctx, load().negf_tally_score_accumulate(ctx, tally, c.ctypes.data, m.ctypes.data))


def negf_current_backward(ctx, tables, tally, mu_p, mu_q, kT, dI, n_sites):
    """Returns (d_onsite, d_eta, stepcap) for all sites (wire after wire)."""
    dI = np.ascontiguousarray(dI, dtype=np.float64)
    dV = np.zeros(max(n_sites, 1))
    dE = np.zeros(max(n_sites, 1))
    st = _check(ctx, load().negf_current_backward(ctx, tables, tally, float(mu_p), float(mu_q),
                                                  float(kT), dI.ctypes.data, dV.ctypes.data,
                                                  dE.ctypes.data), allow=(NEGF_E_STEPCAP,))
    return dV[:n_sites], dE[:n_sites], st == NEGF_E_STEPCAP


def negf_current_backward_rgf(ctx, tables, tally, mu_p, mu_q, kT, dI, n_sites, ckpt_stride=0):
    """As negf_current_backward, by the block-column adjoint (tables with keep_weights; g^L
    and g^R kept every ckpt_stride slices, 0 for the library default)."""
    dI = np.ascontiguousarray(dI, dtype=np.float64)
    dV = np.zeros(max(n_sites, 1))
    dE = np.zeros(max(n_sites, 1))
    st = _check(ctx, load().negf_current_backward_rgf(ctx, tables, tally, float(mu_p), float(mu_q),
                                                      float(kT), dI.ctypes.data, int(ckpt_stride),
                                                      dV.ctypes.data, dE.ctypes.data),
                allow=(NEGF_E_STEPCAP,))
    return dV[:n_sites], dE[:n_sites], st == NEGF_E_STEPCAP


class Plan:
    """Handle of a captured plan plus the arrays it re-reads (kept alive with it)."""

    def __init__(self, handle, keep, n_wires, n_tasks):
        self.handle, self.keep, self.n_wires, self.n_tasks = handle, keep, n_wires, n_tasks


def negf_plan_create(ctx, wires, start_lead, walkers_per_task, mu_p, mu_q, kT, precision="fp32",
                     memspace="host", max_steps=1 << 20, tasks_per_wave=0, waves_in_flight=0,
                     memory_budget=0, walk_blocks_per_sm=0, autotune=True, layout="auto"):
    """Capture build + walk + current of a fixed batch into a CUDA graph; returns a Plan."""
    lib = load()
    keep = []
    arr = _wire_array(wires, memspace, keep)
    bopts = negf_build_opts(PRECISION[precision], 0 if memspace == "host" else 1, 0, 0,
                            LAYOUT[layout])
    ropts = negf_run_opts(int(start_lead), int(tasks_per_wave), 0, int(walkers_per_task), 0,
                          int(max_steps), int(waves_in_flight), int(memory_budget),
                          int(walk_blocks_per_sm), 0)
    out = C.c_void_p()
    _check(ctx, lib.negf_plan_create(ctx, arr, len(wires), C.byref(bopts), C.byref(ropts),
                                     float(mu_p), float(mu_q), float(kT), 1 if autotune else 0,
                                     C.byref(out)))
    if memspace == "host":
        keep = []          # host arrays were read during the call
    return Plan(out, keep, len(wires), lib.negf_plan_num_tasks(out))


def negf_plan_launch(ctx, plan, seed, walker_id_offset=0):
    _check(ctx, load().negf_plan_launch(ctx, plan.handle, int(seed), int(walker_id_offset)))


def negf_plan_result(ctx, plan):
    """dict(I, se, T, T_se, counts, stepcap) of the last launch (synchronises)."""
    nw, nt = max(plan.n_wires, 1), max(plan.n_tasks, 1)
    I, se, T, Tse = np.zeros(nw), np.zeros(nw), np.zeros(nt), np.zeros(nt)
    counts = np.zeros((nt, TALLY_FIELDS), dtype=np.uint64)
    st = _check(ctx, load().negf_plan_result(ctx, plan.handle, I.ctypes.data, se.ctypes.data,
                                             T.ctypes.data, Tse.ctypes.data, counts.ctypes.data),
                allow=(NEGF_E_STEPCAP,))
    return dict(I=I[:plan.n_wires], se=se[:plan.n_wires], T=T[:plan.n_tasks],
                T_se=Tse[:plan.n_tasks], counts=counts[:plan.n_tasks],
                stepcap=st == NEGF_E_STEPCAP)


def negf_plan_get_tuning(plan):
    t = negf_plan_tuning()
    st = load().negf_plan_get_tuning(plan.handle, C.byref(t))
    if st != NEGF_OK:
        raise NegfError(st, "negf_plan_get_tuning")
    return dict(walk_blocks_per_sm=t.walk_blocks_per_sm, chain_warps=t.chain_warps,
                alias_warps=t.alias_warps, tuned=bool(t.tuned), walk_ms=t.walk_ms,
                chain_ms=t.chain_ms, alias_ms=t.alias_ms, walk_slots=t.walk_slots)


def negf_plan_num_waves(plan):
    return load().negf_plan_num_waves(plan.handle)


def negf_plan_device_bytes(plan):
    return load().negf_plan_device_bytes(plan.handle)


def negf_plan_destroy(plan):
    if plan.handle:
        load().negf_plan_destroy(plan.handle)
        plan.handle = None
        plan.keep = []
