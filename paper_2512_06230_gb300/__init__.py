"""Python binding of the GB300 multi-detection GLMB update library.

Thin ctypes marshalling over the C ABI declared in ``include/glmb.h``; every
step of the filter runs in the library's CUDA kernels.  The library is
built in-tree by :func:`build` (sm_103a only).  Importing this module never
falls back to another implementation: if ``libglmb.so`` is missing,
:class:`Filter` raises.

Use::

    import paper_2512_06230_gb300 as glmb
    glmb.build()
    f = glmb.Filter(cfg)                   # cfg: dict of glmb_config fields
    for births, Z in frames:               # births: [(r, mean, cov)], Z: (M, dim_z)
        f.step(births, Z)                  # predict + update + prune (one graph)
        est = f.estimates()                # labels, existence, means, covariances
    f.close()

Several independent scenes step together with :func:`step_batch`; the
learned pair gate is set with :meth:`Filter.set_gate` and trained with
:mod:`paper_2512_06230_gb300.gate`; launch shapes are tuned with
:mod:`paper_2512_06230_gb300.tune`.
"""
from __future__ import annotations

import ctypes as C
import os
import struct
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from typing import Iterable, List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_CSRC = os.path.join(_HERE, "csrc")
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_HERE, "libglmb.so")
HEADER = os.path.join(_ROOT, "include", "glmb.h")
SOURCES = ["kernels_table.cu", "kernels_expand.cu", "kernels_prune.cu", "glmb_api.cu", "gate_mlp.cu",
           "select_static.cu", "select_cluster.cu", "kernels_particle.cu"]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-Xptxas", "-warn-spills"]

STATUS = {0: "GLMB_OK", 1: "GLMB_E_INVALID", 2: "GLMB_E_OOM", 3: "GLMB_E_CAPACITY",
          4: "GLMB_E_CUDA", 5: "GLMB_E_NUMERIC", 6: "GLMB_E_STATE", 7: "GLMB_E_TIMEOUT"}


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the CUDA sources for sm_103a (one TU per process, in parallel)
    and link ``libglmb.so`` next to this file."""
    os.makedirs(_BUILD, exist_ok=True)
    deps = [os.path.join(_CSRC, f) for f in os.listdir(_CSRC)] + [HEADER]
    newest = max(os.path.getmtime(p) for p in deps)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(_BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, *NVCC_FLAGS, "-c", os.path.join(_CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp,
                        *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


# --------------------------------------------------------------------------
# C structs (layouts of include/glmb.h)
# --------------------------------------------------------------------------
# device allocation hook of glmb_config
DEV_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
DEV_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class GlmbConfig(C.Structure):
    _fields_ = [("dim_x", C.c_int32), ("dim_z", C.c_int32), ("dt", C.c_float), ("q", C.c_double),
                ("R", C.c_double * 9), ("p_s", C.c_double), ("p_d", C.c_double),
                ("lambda_d", C.c_double), ("clutter_rate", C.c_double), ("volume", C.c_double),
                ("gate", C.c_double), ("h_max", C.c_int32), ("h_up", C.c_int32), ("tau", C.c_double),
                ("seed", C.c_uint64), ("score_mode", C.c_int32), ("max_tracks", C.c_int32),
                ("max_meas", C.c_int32), ("max_births", C.c_int32), ("max_pairs", C.c_int64),
                ("stream", C.c_void_p), ("max_components", C.c_int64),
                ("dev_alloc", DEV_ALLOC_FN), ("dev_free", DEV_FREE_FN), ("alloc_ctx", C.c_void_p),
                ("model", C.c_int32), ("n_particles", C.c_int32), ("sigma_a", C.c_double),
                ("sigma_w", C.c_double), ("ess_frac", C.c_double)]


class GlmbBirth(C.Structure):
    _fields_ = [("r", C.c_double), ("mean", C.c_double * 6), ("cov", C.c_double * 36)]


class GlmbTrack(C.Structure):
    _fields_ = [("label_k", C.c_uint32), ("label_b", C.c_uint32), ("r", C.c_double),
                ("mean", C.c_double * 6), ("cov", C.c_double * 36)]


class GlmbInfo(C.Structure):
    _fields_ = [("frame", C.c_int32), ("n_hyp", C.c_int32), ("n_entries", C.c_int64),
                ("n_components", C.c_int32), ("n_meas", C.c_int32), ("n_pairs", C.c_int64),
                ("n_children", C.c_int64), ("n_unique", C.c_int64), ("n_updates", C.c_int32),
                ("n_fp64_chol", C.c_int32), ("n_launches", C.c_int64),
                ("n_graph_captures", C.c_int64), ("n_graph_launches", C.c_int64),
                ("n_redo", C.c_int64), ("expand_smem_bytes", C.c_int32),
                ("expand_ctas_per_sm", C.c_int32), ("expand_plan_T", C.c_int32),
                ("expand_plan_K", C.c_int32), ("expand_plan_M", C.c_int32),
                ("expand_threads", C.c_int32), ("graph_capture_ms", C.c_double),
                ("n_pairs_pregate", C.c_int64), ("n_draw_overflow", C.c_int64)]


class GlmbTuning(C.Structure):
    """Launch shapes (glmb_tuning); results do not depend on them."""
    _fields_ = [("thread_warps_per_sm", C.c_int32), ("draw_threads", C.c_int32),
                ("warp_cta_warps", C.c_int32), ("stage_threads", C.c_int32)]


class GlmbFrameIn(C.Structure):
    """One scene's frame for glmb_step_batch."""
    _fields_ = [("births", C.c_void_p), ("n_births", C.c_int32), ("z_is_device", C.c_int32),
                ("Z", C.c_void_p), ("M", C.c_int32), ("pad", C.c_int32)]


# NumPy views of the ABI records (same layout as the C structs)
BIRTH_DTYPE = np.dtype([("r", "<f8"), ("mean", "<f8", 6), ("cov", "<f8", 36)])
TRACK_DTYPE = np.dtype([("label_k", "<u4"), ("label_b", "<u4"), ("r", "<f8"), ("mean", "<f8", 6),
                        ("cov", "<f8", 36)])

_lib = None


def declared_functions() -> List[str]:
    """Names of the entry points declared in include/glmb.h."""
    import re
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:glmb_status|const char\*)\s+(glmb_\w+)\s*\(", text,
                                 re.M)))


def load() -> C.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libglmb.so is not built: run paper_2512_06230_gb300.build() "
                           "(needs nvcc); there is no fallback implementation")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    I, L = C.c_int, C.c_int64
    sig = {
        "glmb_create": [P, P], "glmb_destroy": [P], "glmb_reset": [P],
        "glmb_predict": [P, P, I], "glmb_update": [P, P, I, I], "glmb_prune": [P],
        "glmb_estimates": [P, P, I, P, P, I], "glmb_meas_assoc": [P, P, I],
        "glmb_get_info": [P, P], "glmb_export_state": [P, P, C.c_size_t, P],
        "glmb_import_state": [P, P, C.c_size_t],
        "glmb_get_hypotheses": [P, P, P, P, P, P, P, I, L, P],
        "glmb_get_parents": [P, P, P, I, L, P],
        "glmb_get_components": [P, P, P, P, P, P, P, P, I, P],
        "glmb_get_pairs": [P, P, P, P, P, P, I, L, P],
        "glmb_get_children": [P, P, P, P, L, P],
        "glmb_set_profiling": [P, C.c_uint], "glmb_get_timing": [P, P, P, I],
        "glmb_get_retained": [P, P, P, I, P],
        "glmb_step": [P, P, I, P, I, I], "glmb_set_step_estimates": [P, I], "glmb_set_launch_options": [P, C.c_uint],
        "glmb_step_enqueue": [P, P, I, P, I, I], "glmb_step_finish": [P],
        "glmb_step_batch": [P, I, P, P], "glmb_set_tuning": [P, P], "glmb_get_tuning": [P, P],
        "glmb_set_gate": [P, P, C.c_float, I], "glmb_gate_features": [P, P, L, P],
        "glmb_gate_logits": [P, P, L, P], "glmb_gate_usage": [P, P, L, P, I, P, P],
        "glmb_mlp_forward": [P, P, L, P, P, P], "glmb_mlp_backward": [P, P, P, P, L, P, P, P, P],
        "glmb_mlp_adam": [P, P, P, P, I, C.c_float, C.c_float, C.c_float, C.c_float, P],
        "glmb_set_wait_test": [I, C.c_longlong],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.glmb_last_error.argtypes = [P]
    lib.glmb_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def torch_allocator_hooks(device=None):
    """(dev_alloc, dev_free) callbacks over torch.cuda's caching allocator.
    The blocks are taken on torch's current stream of `device`; the library
    returns a block only after its own stream has finished with it."""
    import torch

    dev = torch.cuda.current_device() if device is None else device

    def _alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device=dev)
        except RuntimeError:
            return None

    def _free(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    return DEV_ALLOC_FN(_alloc), DEV_FREE_FN(_free)


WAIT_TEST_OFF, WAIT_TEST_SCAN, WAIT_TEST_GATE = 0, 1, 2


def set_wait_test(mode: int, limit: int = 0) -> None:
    """Failure-detection test hook (glmb_set_wait_test): make one bounded
    device wait run out (WAIT_TEST_SCAN, WAIT_TEST_GATE) after `limit`, or
    restore the normal limits (WAIT_TEST_OFF)."""
    st = load().glmb_set_wait_test(int(mode), int(limit))
    if st != 0:
        raise GlmbError(st, "glmb_set_wait_test rejected its arguments")


class GlmbError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def make_config(cfg: dict, stream: Optional[int] = None) -> GlmbConfig:
    c = GlmbConfig()
    c.dim_x, c.dim_z = int(cfg["dim_x"]), int(cfg["dim_z"])
    c.dt, c.q = float(cfg["dt"]), float(cfg["q"])
    d = c.dim_z
    R = np.asarray(cfg["R"], dtype=np.float64).reshape(d, d).ravel()
    for i in range(d * d):
        c.R[i] = R[i]
    c.p_s, c.p_d, c.lambda_d = float(cfg["p_s"]), float(cfg["p_d"]), float(cfg["lambda_d"])
    c.clutter_rate, c.volume, c.gate = float(cfg["clutter_rate"]), float(cfg["volume"]), float(cfg["gate"])
    c.h_max, c.h_up, c.tau = int(cfg["h_max"]), int(cfg["h_up"]), float(cfg["tau"])
    c.seed = int(cfg["seed"]) & 0xFFFFFFFFFFFFFFFF
    c.score_mode = int(cfg.get("score_mode", 0))
    c.max_tracks = int(cfg.get("max_tracks", 0))
    c.max_meas = int(cfg.get("max_meas", 0))
    c.max_births = int(cfg.get("max_births", 0))
    c.max_pairs = int(cfg.get("max_pairs", 0))
    c.max_components = int(cfg.get("max_components", 0))
    c.stream = stream
    c.model = int(cfg.get("model", 0))
    c.n_particles = int(cfg.get("n_particles", 0))
    c.sigma_a = float(cfg.get("sigma_a", 0.0))
    c.sigma_w = float(cfg.get("sigma_w", 0.0))
    c.ess_frac = float(cfg.get("ess_frac", 0.0))
    return c


def births_array(births, dim_x: int) -> np.ndarray:
    """glmb_birth records (BIRTH_DTYPE) from (r, mean, cov) tuples."""
    arr = np.zeros(len(births), BIRTH_DTYPE)
    for j, (r, m, P) in enumerate(births):
        arr[j]["r"] = r
        arr[j]["mean"][:dim_x] = np.asarray(m, np.float64).reshape(dim_x)
        arr[j]["cov"][: dim_x * dim_x] = np.asarray(P, np.float64).reshape(dim_x * dim_x)
    return arr


def pack_state(frame: int, logw, uid, tracks, dim_x: int, n_particles: int = 0) -> bytes:
    """State buffer of include/glmb.h from per-hypothesis track lists of
    (label_k, label_b, mean, cov), with the particle model (label_k,
    label_b, mean, cov, x[P][5], logw[P]) (version 2)."""
    H = len(logw)
    n = sum(len(t) for t in tracks)
    out = [struct.pack("<IIiiiiq", 0x424D4C47, 2 if n_particles else 1, dim_x, frame, H, 0, n)]
    for h in range(H):
        out.append(struct.pack("<dQii", float(logw[h]), int(uid[h]), len(tracks[h]), 0))
    for tr in tracks:
        for rec in tr:
            k, b, m, P = rec[:4]
            out.append(struct.pack("<II", int(k), int(b)))
            out.append(np.asarray(m, dtype="<f8").reshape(dim_x).tobytes())
            out.append(np.asarray(P, dtype="<f8").reshape(dim_x, dim_x).tobytes())
            if n_particles:
                out.append(np.asarray(rec[4], dtype="<f8").reshape(n_particles, 5).tobytes())
                out.append(np.asarray(rec[5], dtype="<f8").reshape(n_particles).tobytes())
    return b"".join(out)


def unpack_state(buf: bytes, n_particles: int = 0):
    magic, ver, dx, frame, H, _, n = struct.unpack_from("<IIiiiiq", buf, 0)
    off = struct.calcsize("<IIiiiiq")
    logw, uid, ntr = [], [], []
    for _ in range(H):
        lw, u, nt, _ = struct.unpack_from("<dQii", buf, off)
        off += struct.calcsize("<dQii")
        logw.append(lw)
        uid.append(u)
        ntr.append(nt)
    tracks = []
    for nt in ntr:
        tr = []
        for _ in range(nt):
            k, b = struct.unpack_from("<II", buf, off)
            off += 8
            m = np.frombuffer(buf, "<f8", dx, off).copy()
            off += 8 * dx
            P = np.frombuffer(buf, "<f8", dx * dx, off).reshape(dx, dx).copy()
            off += 8 * dx * dx
            if ver == 2:
                x = np.frombuffer(buf, "<f8", 5 * n_particles, off).reshape(n_particles, 5).copy()
                off += 40 * n_particles
                pw = np.frombuffer(buf, "<f8", n_particles, off).copy()
                off += 8 * n_particles
                tr.append((k, b, m, P, x, pw))
            else:
                tr.append((k, b, m, P))
        tracks.append(tr)
    return frame, np.array(logw), np.array(uid, dtype=np.uint64), tracks


class Filter:
    """One GLMB filter on the current CUDA device (see include/glmb.h)."""

    def __init__(self, cfg: dict, stream: Optional[int] = None, allocator=None):
        """allocator="torch": the handle's device memory comes from PyTorch's
        caching allocator (glmb_config.dev_alloc / dev_free); a pair of
        callables (alloc(nbytes) -> device address or None, free(address))
        routes it through the caller's own functions."""
        self.lib = load()
        self.cfg = dict(cfg)
        self._c = make_config(cfg, stream)
        if allocator == "torch":
            self._hooks = torch_allocator_hooks()
            self._c.dev_alloc, self._c.dev_free = self._hooks
        elif isinstance(allocator, tuple) and len(allocator) == 2:
            fa, ff = allocator
            self._hooks = (DEV_ALLOC_FN(lambda nbytes, ctx: fa(int(nbytes))),
                           DEV_FREE_FN(lambda ptr, ctx: ff(ptr)))
            self._c.dev_alloc, self._c.dev_free = self._hooks
        elif allocator is not None:
            raise ValueError(f"unknown allocator {allocator!r}")
        self.dx, self.dz = self._c.dim_x, self._c.dim_z
        h = C.c_void_p()
        st = self.lib.glmb_create(C.byref(self._c), C.byref(h))
        if st != 0:
            raise GlmbError(st, "glmb_create rejected the configuration")
        self.h = h
        self.M = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.glmb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != 0:
            raise GlmbError(st, self.lib.glmb_last_error(self.h).decode())

    # ---- filter steps ----
    def reset(self):
        self._check(self.lib.glmb_reset(self.h))

    def _births(self, births):
        if isinstance(births, np.ndarray) and births.dtype == BIRTH_DTYPE:
            return np.ascontiguousarray(births)
        return births_array(births, self.dx)

    def predict(self, births):
        arr = self._births(births)
        self._check(self.lib.glmb_predict(self.h, _ptr(arr), len(births)))

    def _dev_z(self, Z):
        """Pointer and row count of detections in device memory: a CUDA
        tensor (torch) of shape (M, dim_z), float32, contiguous.  Anything
        else is refused here, before the kernels could read it as such."""
        if not getattr(Z, "is_cuda", False):
            raise TypeError("device detections: a CUDA tensor is required")
        if not Z.is_floating_point() or Z.element_size() != 4 or Z.is_complex():
            raise TypeError(f"device detections: float32 required, got {Z.dtype}")
        if Z.dim() != 2 or (Z.shape[1] != self.dz and Z.shape[0] > 0):
            raise ValueError(f"device detections: shape (M, {self.dz}) required, got {tuple(Z.shape)}")
        if not Z.is_contiguous():
            raise ValueError("device detections: a contiguous tensor is required")
        return C.c_void_p(Z.data_ptr()), int(Z.shape[0])

    def update(self, Z, device: bool = False):
        if device:
            zp, M = self._dev_z(Z)
            self.M = M
            self._check(self.lib.glmb_update(self.h, zp, M, 1))
            return
        Zf = np.ascontiguousarray(Z, dtype=np.float32).reshape(-1, self.dz)
        self.M = len(Zf)
        self._check(self.lib.glmb_update(self.h, _ptr(Zf), len(Zf), 0))

    def prune(self):
        self._check(self.lib.glmb_prune(self.h))

    def _frame_args(self, births, Z, device):
        arr = self._births(births)
        if device:
            zp, M = self._dev_z(Z)
            return arr, len(births), zp, M, 1, None
        Zf = np.ascontiguousarray(Z, dtype=np.float32).reshape(-1, self.dz)
        return arr, len(births), _ptr(Zf), len(Zf), 0, Zf

    def step_enqueue(self, births, Z, device: bool = False):
        """Launches one frame (glmb_step_enqueue); step_finish completes it.
        Host arrays are kept alive until then."""
        arr, nb, zp, M, dev, keep = self._frame_args(births, Z, device)
        self.M = M
        self._inflight = (arr, keep, Z)
        self._check(self.lib.glmb_step_enqueue(self.h, _ptr(arr), nb, zp, M, dev))

    def step_finish(self):
        self._check(self.lib.glmb_step_finish(self.h))
        self._inflight = None

    def tuning(self) -> dict:
        t = GlmbTuning()
        self._check(self.lib.glmb_get_tuning(self.h, C.byref(t)))
        return {k: getattr(t, k) for k, _ in GlmbTuning._fields_}

    def set_tuning(self, **kw):
        cur = self.tuning()
        cur.update(kw)
        t = GlmbTuning(**cur)
        self._check(self.lib.glmb_set_tuning(self.h, C.byref(t)))

    def step(self, births, Z, device: bool = False):
        """One frame in one call (glmb_step: a replayed CUDA graph)."""
        arr = self._births(births)
        if device:
            zp, M = self._dev_z(Z)
            self.M = M
            self._check(self.lib.glmb_step(self.h, _ptr(arr), len(births), zp, M, 1))
            return
        Zf = np.ascontiguousarray(Z, dtype=np.float32).reshape(-1, self.dz)
        self.M = len(Zf)
        self._check(self.lib.glmb_step(self.h, _ptr(arr), len(births), _ptr(Zf), len(Zf), 0))

    # ---- outputs ----
    def estimates(self, cap: int = 4096, pmf_cap: int = 4096):
        """MAP tracks (labels, existence, mean, cov) and the cardinality pmf."""
        # the output buffers and their pointers are kept between calls (this
        # runs once per frame; building ctypes pointers costs microseconds)
        buf = getattr(self, "_est_buf", None)
        if buf is None or len(buf[0]) < cap or len(buf[1]) < pmf_cap:
            o, q, n = np.zeros(cap, TRACK_DTYPE), np.zeros(pmf_cap), C.c_int()
            buf = (o, q, _ptr(o), _ptr(q), n, C.byref(n))
            self._est_buf = buf
        out, pmf, p_out, p_pmf, n, n_ref = buf
        self._check(self.lib.glmb_estimates(self.h, p_out, cap, n_ref, p_pmf, pmf_cap))
        k, dx = n.value, self.dx
        t = out[:k].copy()
        # every field is a view of this call's own copy of the records;
        # labels: (k, 2) of (label_k, label_b), the records' first two words
        words = t.view(np.uint32).reshape(k, TRACK_DTYPE.itemsize // 4)
        return dict(n=k, labels=words[:, :2], r=t["r"], mean=t["mean"][:, :dx],
                    cov=t["cov"][:, : dx * dx].reshape(k, dx, dx), pmf=pmf[:pmf_cap].copy())

    STAGES = ("predict", "table", "expand", "select", "materialize", "update_gc", "estimates")

    OPT_STAGE_GLOBAL, OPT_DRAW_WARP, OPT_DRAW_THREAD, OPT_STAGE_SHARED = 1, 2, 4, 8
    OPT_STAGE_SCRATCH_ROWS, OPT_STAGE_SCRATCH_NONE, OPT_WARP_GROUPS = 16, 32, 64

    # ---- learned pair gate ----
    GATE_OFF, GATE_PRUNE, GATE_SCORE = 0, 1, 2

    def set_gate(self, params=None, threshold: float = 0.0, mode: int = 1):
        """Learned gate for the following updates (params: GATE_NPARAM
        float32 values; mode GATE_PRUNE drops pairs whose logit < threshold,
        GATE_SCORE only scores them; None switches it off)."""
        if params is None:
            self._check(self.lib.glmb_set_gate(self.h, None, C.c_float(0.0), self.GATE_OFF))
            return
        p = np.ascontiguousarray(params, np.float32).reshape(-1)
        if p.size != GATE_NPARAM:
            raise ValueError(f"gate parameters: {p.size} values, need {GATE_NPARAM}")
        self._check(self.lib.glmb_set_gate(self.h, _ptr(p), C.c_float(threshold), int(mode)))

    def gate_features(self) -> np.ndarray:
        """Raw features (K x 5) of the last update's pairs before the gate."""
        n = C.c_int64()
        self.lib.glmb_gate_features(self.h, None, 0, C.byref(n))
        X = np.zeros((max(n.value, 1), 5), np.float32)
        self._check(self.lib.glmb_gate_features(self.h, _ptr(X), X.shape[0], C.byref(n)))
        return X[: n.value]

    def gate_logits(self) -> np.ndarray:
        n = C.c_int64()
        self.lib.glmb_gate_logits(self.h, None, 0, C.byref(n))
        z = np.zeros(max(n.value, 1), np.float32)
        self._check(self.lib.glmb_gate_logits(self.h, _ptr(z), z.size, C.byref(n)))
        return z[: n.value]

    def gate_usage(self):
        """(used[K] uint8, hyp_flag[H] uint8) of the last pruned frame."""
        K, H = C.c_int64(), C.c_int()
        self.lib.glmb_gate_usage(self.h, None, 0, None, 0, C.byref(K), C.byref(H))
        used = np.zeros(max(K.value, 1), np.uint8)
        flag = np.zeros(max(H.value, 1), np.uint8)
        self._check(self.lib.glmb_gate_usage(self.h, _ptr(used), used.size, _ptr(flag), flag.size,
                                             C.byref(K), C.byref(H)))
        return used[: K.value], flag[: H.value]

    def set_launch_options(self, opts: int = 0):
        self._check(self.lib.glmb_set_launch_options(self.h, int(opts)))

    def set_step_estimates(self, on: bool = True):
        self._check(self.lib.glmb_set_step_estimates(self.h, 1 if on else 0))

    def set_profiling(self, stages: Iterable[str] = ()):
        mask = 0
        for s in stages:
            mask |= 1 << self.STAGES.index(s)
        self._check(self.lib.glmb_set_profiling(self.h, mask))

    def timing(self) -> dict:
        n = len(self.STAGES)
        ms = np.zeros(n)
        calls = np.zeros(n, np.int64)
        self._check(self.lib.glmb_get_timing(self.h, _ptr(ms), _ptr(calls), n))
        return {s: (float(ms[i]), int(calls[i])) for i, s in enumerate(self.STAGES)}

    def meas_assoc(self):
        r = np.zeros(max(self.M, 1))
        self._check(self.lib.glmb_meas_assoc(self.h, _ptr(r), len(r)))
        return r[: self.M]

    def info(self) -> dict:
        inf = GlmbInfo()
        self._check(self.lib.glmb_get_info(self.h, C.byref(inf)))
        return {k: getattr(inf, k) for k, _ in GlmbInfo._fields_}

    def export_state(self) -> bytes:
        n = C.c_size_t()
        self._check(self.lib.glmb_export_state(self.h, None, 0, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(self.lib.glmb_export_state(self.h, buf, n.value, C.byref(n)))
        return buf.raw[: n.value]

    def import_state(self, buf: bytes):
        self._check(self.lib.glmb_import_state(self.h, buf, len(buf)))

    def hypotheses(self):
        inf = self.info()
        H, E = inf["n_hyp"], inf["n_entries"]
        logw = np.zeros(H)
        uid = np.zeros(H, np.uint64)
        ptr = np.zeros(H + 1, np.uint32)
        lk = np.zeros(max(E, 1), np.uint32)
        lb = np.zeros(max(E, 1), np.uint32)
        theta = np.zeros((H, max(self.M, 1)), np.uint16)
        n = C.c_int()
        self._check(self.lib.glmb_get_hypotheses(self.h, _ptr(logw), _ptr(uid), _ptr(ptr), _ptr(lk),
                                                 _ptr(lb), _ptr(theta), H, max(E, 1), C.byref(n)))
        return dict(logw=logw, uid=uid, ptr=ptr, label_k=lk[:E], label_b=lb[:E],
                    theta=theta[:, : self.M])

    def retained(self):
        """Child indices (parent * h_up + draw) and renormalised log-weights
        of the hypotheses kept by the last prune."""
        n = C.c_int()
        self.lib.glmb_get_retained(self.h, None, None, 0, C.byref(n))
        k = n.value
        idx = np.zeros(max(k, 1), np.int64)
        lw = np.zeros(max(k, 1))
        self._check(self.lib.glmb_get_retained(self.h, _ptr(idx), _ptr(lw), max(k, 1), C.byref(n)))
        return idx[:k], lw[:k]

    def parents(self):
        n = C.c_int()
        self.lib.glmb_get_parents(self.h, None, None, 0, 0, C.byref(n))
        H = n.value
        cap = (H + 1) * (self._c.max_tracks or 256) + 16
        ptr = np.zeros(H + 1, np.uint32)
        comp = np.zeros(cap, np.uint32)
        self._check(self.lib.glmb_get_parents(self.h, _ptr(ptr), _ptr(comp), H, cap, C.byref(n)))
        return ptr, comp[: ptr[H]]

    def components(self):
        n = C.c_int()
        self.lib.glmb_get_components(self.h, None, None, None, None, None, None, None, 0, C.byref(n))
        T, dx = n.value, self.dx
        lk = np.zeros(max(T, 1), np.uint32)
        lb = np.zeros(max(T, 1), np.uint32)
        mean = np.zeros((max(T, 1), dx))
        cov = np.zeros((max(T, 1), dx, dx))
        p = np.zeros(max(T, 1))
        dp = np.zeros(max(T, 1))
        ld = np.zeros(max(T, 1))
        self._check(self.lib.glmb_get_components(self.h, _ptr(lk), _ptr(lb), _ptr(mean), _ptr(cov),
                                                 _ptr(p), _ptr(dp), _ptr(ld), max(T, 1), C.byref(n)))
        return dict(label_k=lk[:T], label_b=lb[:T], mean=mean[:T], cov=cov[:T], p=p[:T],
                    dprob=dp[:T], logdetS=ld[:T])

    def pairs(self):
        T = self.components()["p"].shape[0]
        K = C.c_int64()
        self.lib.glmb_get_pairs(self.h, None, None, None, None, None, 0, 0, C.byref(K))
        k = K.value
        ptr = np.zeros(T + 1, np.uint32)
        meas = np.zeros(max(k, 1), np.uint32)
        logC = np.zeros(max(k, 1), np.float32)
        q = np.zeros(max(k, 1), np.float32)
        e = np.zeros((max(k, 1), self.dz), np.float32)
        self._check(self.lib.glmb_get_pairs(self.h, _ptr(ptr), _ptr(meas), _ptr(logC), _ptr(q), _ptr(e),
                                            T + 1, max(k, 1), C.byref(K)))
        return dict(ptr=ptr, meas=meas[:k], logC=logC[:k], q=q[:k], e=e[:k])

    def children(self):
        n = C.c_int64()
        self.lib.glmb_get_children(self.h, None, None, None, 0, C.byref(n))
        k = n.value
        logw = np.zeros(max(k, 1))
        st = np.zeros(max(k, 1), np.int8)
        na = np.zeros(max(k, 1), np.uint16)
        self._check(self.lib.glmb_get_children(self.h, _ptr(logw), _ptr(st), _ptr(na), max(k, 1),
                                               C.byref(n)))
        return dict(logw=logw[:k], status=st[:k], n_alive=na[:k])


GATE_NPARAM = 8779
GATE_NTRAIN = 8769


def _tptr(t):
    return C.c_void_p(t.data_ptr())


def _stream(stream, t):
    """The CUDA stream to enqueue on: the given one, else torch's current
    stream on the device of tensor t (so the call orders with torch's own
    work on its tensors)."""
    if stream is not None:
        return C.c_void_p(stream)
    import torch
    return C.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def mlp_forward(params, X, err, stream=None):
    """Logits of the raw feature rows X (torch float32 (n, 5), CUDA) through
    glmb_mlp_forward; err: a zeroed CUDA uint32/int32 tensor of one element
    that receives 256 if a tensor-core wait ran out of time."""
    import torch
    n = int(X.shape[0])
    out = torch.empty(n, dtype=torch.float32, device=X.device)
    st = load().glmb_mlp_forward(_tptr(params), _tptr(X), n, _tptr(out), _tptr(err), _stream(stream, X))
    if st:
        raise GlmbError(st, "mlp_forward")
    return out


def mlp_backward(params, X, y, wt, grad, loss, err, stream=None):
    """Fills grad (GATE_NPARAM float32) and loss (one float64) on the device."""
    n = int(X.shape[0])
    st = load().glmb_mlp_backward(_tptr(params), _tptr(X), _tptr(y), _tptr(wt), n, _tptr(grad), _tptr(loss),
                                  _tptr(err), _stream(stream, X))
    if st:
        raise GlmbError(st, "mlp_backward")


def mlp_adam(params, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    st = load().glmb_mlp_adam(_tptr(params), _tptr(grad), _tptr(m), _tptr(v), int(step), C.c_float(lr),
                              C.c_float(beta1), C.c_float(beta2), C.c_float(eps), _stream(stream, params))
    if st:
        raise GlmbError(st, "mlp_adam")


def step_batch(filters, frames, device: bool = False):
    """One frame of several independent filters (glmb_step_batch): all are
    launched, then all completed, so that their graphs overlap on the GPU.
    frames: a list of (births, Z) per filter.  Raises on the first error."""
    n = len(filters)
    if n == 0:
        return
    lib = filters[0].lib
    hs = (C.c_void_p * n)(*[f.h for f in filters])
    ins = (GlmbFrameIn * n)()
    keep = []
    for i, (f, (births, Z)) in enumerate(zip(filters, frames)):
        arr, nb, zp, M, dev, zf = f._frame_args(births, Z, device)
        keep.append((arr, zf, Z))
        f.M = M
        ins[i] = GlmbFrameIn(arr.ctypes.data if len(arr) else None, nb, dev, zp, M, 0)
    st = (C.c_int * n)()
    rc = lib.glmb_step_batch(hs, n, ins, st)
    if rc != 0:
        bad = next(i for i in range(n) if st[i] != 0)
        raise GlmbError(st[bad], f"scene {bad}: " + lib.glmb_last_error(filters[bad].h).decode())
