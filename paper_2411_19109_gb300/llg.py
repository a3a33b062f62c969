"""ctypes binding of the C ABI in include/llg.h.

Argument marshalling only: every step of the forward pass, the adjoint and
the level-set update runs in the CUDA library.  Functions carry the C names
(llg_create, llg_forward, llg_adjoint, levelset_step, llg_field, llg_query,
llg_launch_count, llg_last_error, llg_destroy, llg_schedule,
llg_padded_extents); `Solver` bundles them for torch tensors.

Loading fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np

from . import build as _build

c_int, c_double, c_ll, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_void_p
_PD = ctypes.POINTER(c_double)

LLG_OK, LLG_EINVAL, LLG_ENOMEM, LLG_ECUDA, LLG_ETIMEOUT, LLG_ENONFINITE, LLG_ESTATE = range(7)
LLG_J_PORT, LLG_J_ENERGY_AREA, LLG_J_SPECTRAL, LLG_J_CURVE = 0, 1, 2, 3
LLG_FP32, LLG_FP64 = 0, 1
LLG_CKPT_STORE_ALL, LLG_CKPT_PERIODIC, LLG_CKPT_BINOMIAL = 0, 1, 2
LLG_INT_RK4, LLG_INT_DOPRI5 = 0, 1
LLG_SPEC_WORKING, LLG_SPEC_DFLOAT = 0, 1
LLG_TUNE_DEFAULT, LLG_TUNE_MEASURE, LLG_TUNE_GIVEN = 0, 1, 2
LLG_RECORD_STAGES, LLG_RECORD_STATES = 0, 1

EXPORTED = ("llg_create", "llg_forward", "llg_adjoint", "levelset_step", "llg_field", "llg_query",
            "llg_launch_count", "llg_kernel_time", "llg_last_error", "llg_destroy", "llg_schedule",
            "llg_padded_extents", "llg_abi_version", "llg_field_noalloc", "llg_rbf_workspace_bytes",
            "llg_rbf_phi", "llg_rbf_grad", "llg_adam_step", "llg_fp64_fma_rate", "llg_adaptive_steps",
            "llg_launch_config")


class llg_rbf(ctypes.Structure):
    """RBF level-set layout (C struct llg_rbf)."""
    _fields_ = [("nx", c_int), ("ny", c_int), ("dx", c_double), ("dy", c_double), ("box", c_int * 4),
                ("nrx", c_int), ("nry", c_int), ("p", c_double)]


class llg_problem(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int),
                ("dx", c_double), ("dy", c_double), ("dz", c_double),
                ("Ms", c_double), ("A", c_double), ("Ku", c_double), ("ku", c_double * 3),
                ("alpha", c_double), ("alpha_edge", c_double),
                ("absorb_nodes", c_int), ("absorb_x", c_int), ("absorb_y", c_int),
                ("B_bias", c_double * 3), ("b_rf", c_double), ("f_rf", c_double),
                ("rf_dir", c_double * 3), ("src", c_int * 4),
                ("dt", c_double), ("nsteps", c_ll), ("sigmoid_a", c_double),
                ("objective", c_int), ("comp", c_int), ("power", c_int),
                ("boxes", (c_int * 4) * 2), ("weights", c_double * 2), ("n_from", c_ll),
                ("area_target", c_double), ("penalty_w", c_double), ("nfreq", c_int), ("freqs", c_double * 8),
                ("drive", _PD), ("nsample", c_int), ("sample_step", ctypes.POINTER(c_ll)),
                ("sample_target", _PD), ("sample_weight", _PD), ("centre_w", c_double),
                ("centre_target", c_double * 2)]


class llg_launch(ctypes.Structure):
    _fields_ = [("col_lanes", c_int), ("col_blocks", c_int), ("adj_blocks", c_int), ("groups", c_int),
                ("adj_split", c_int)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class llg_options(ctypes.Structure):
    _fields_ = [("precision", c_int), ("ckpt", c_int), ("seg_len", c_int), ("use_graph", c_int),
                ("tune", c_int), ("time_kernels", c_int), ("integrator", c_int),
                ("rtol", c_double), ("atol", c_double), ("adj_spectral", c_int), ("launch", llg_launch),
                ("record", c_int)]


class LLGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"LLG status {status}: {msg}")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load (building first if needed) the in-tree CUDA library."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"CUDA library {_build.LIB} is missing; run build() first")
    lib = ctypes.CDLL(_build.LIB)
    P = ctypes.POINTER
    lib.llg_create.argtypes = [P(llg_problem), c_int, P(llg_options), c_void_p, P(c_void_p)]
    lib.llg_forward.argtypes = [c_void_p, c_void_p, c_void_p, P(c_double), c_void_p]
    lib.llg_adjoint.argtypes = [c_void_p, _PD, c_void_p, c_void_p]
    lib.llg_launch_config.argtypes = [c_void_p, ctypes.POINTER(llg_launch), _PD]
    lib.llg_launch_config.restype = c_int
    lib.levelset_step.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_double]
    lib.llg_field.argtypes = [c_void_p, c_void_p, c_void_p, c_double, c_int, c_void_p]
    lib.llg_query.argtypes = [c_void_p, P(ctypes.c_size_t), P(c_double)]
    lib.llg_launch_count.argtypes = [c_void_p]
    lib.llg_launch_count.restype = c_ll
    lib.llg_kernel_time.argtypes = [c_void_p, c_int, P(c_ll), P(c_double)]
    lib.llg_kernel_time.restype = c_int
    lib.llg_last_error.argtypes = [c_void_p]
    lib.llg_last_error.restype = ctypes.c_char_p
    lib.llg_destroy.argtypes = [c_void_p]
    lib.llg_destroy.restype = None
    lib.llg_schedule.argtypes = [c_ll, c_int, c_int, P(c_ll), c_ll, P(c_ll)]
    lib.llg_schedule.restype = c_ll
    lib.llg_padded_extents.argtypes = [c_int, c_int, P(c_int), P(c_int)]
    lib.llg_abi_version.restype = c_int
    lib.llg_field_noalloc.argtypes = [P(llg_problem), c_void_p, c_void_p, c_double, c_int, c_void_p, c_void_p,
                                      P(ctypes.c_char_p)]
    lib.llg_field_noalloc.restype = c_int
    lib.llg_rbf_workspace_bytes.argtypes = [P(llg_rbf)]
    lib.llg_rbf_workspace_bytes.restype = ctypes.c_size_t
    lib.llg_rbf_phi.argtypes = [P(llg_rbf), c_void_p, c_void_p, c_int, c_void_p, c_void_p]
    lib.llg_rbf_phi.restype = c_int
    lib.llg_rbf_grad.argtypes = [P(llg_rbf), c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p]
    lib.llg_rbf_grad.restype = c_int
    lib.llg_adam_step.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_ll, c_double, c_double, c_double,
                                  c_double, c_void_p]
    lib.llg_adam_step.restype = c_int
    lib.llg_adaptive_steps.argtypes = [c_void_p, c_int, P(c_double), P(c_double), c_ll, P(c_ll)]
    lib.llg_adaptive_steps.restype = c_int
    lib.llg_fp64_fma_rate.argtypes = [c_int, P(c_double), P(c_double), c_void_p]
    lib.llg_fp64_fma_rate.restype = c_int
    for f in ("llg_create", "llg_forward", "llg_adjoint", "levelset_step", "llg_field", "llg_query"):
        getattr(lib, f).restype = c_int
    _lib = lib
    return lib


def to_struct(p) -> llg_problem:
    """llg_problem from any object with the fields of workloads.Problem."""
    s = llg_problem()
    s.nx, s.ny, s.nz = p.nx, p.ny, p.nz
    s.dx, s.dy, s.dz = p.dx, p.dy, p.dz
    s.Ms, s.A, s.Ku = p.Ms, p.A, p.Ku
    s.ku[:] = list(p.ku)
    s.alpha, s.alpha_edge = p.alpha, p.alpha_edge
    s.absorb_nodes, s.absorb_x, s.absorb_y = p.absorb_nodes, p.absorb_x, p.absorb_y
    s.B_bias[:] = list(p.B_bias)
    s.b_rf, s.f_rf = p.b_rf, p.f_rf
    s.rf_dir[:] = list(p.rf_dir)
    s.src[:] = list(p.src)
    s.dt, s.nsteps, s.sigmoid_a = p.dt, p.nsteps, p.sigmoid_a
    s.objective, s.comp, s.power = p.objective, p.comp, p.power
    for b in range(2):
        s.boxes[b][:] = list(p.boxes[b])
    s.weights[:] = list(p.weights)
    s.n_from = p.n_from
    s.area_target, s.penalty_w = p.area_target, p.penalty_w
    fq = list(getattr(p, "freqs", ()))
    s.nfreq = len(fq)
    s.freqs[:min(len(fq), 8)] = fq[:8]
    # host arrays: kept alive on the struct (the library copies them at create)
    keep = []
    drive = getattr(p, "drive", None)
    if drive is not None:
        a = (c_double * len(drive))(*drive)
        keep.append(a)
        s.drive = ctypes.cast(a, _PD)
    steps = list(getattr(p, "sample_steps", ()))
    if steps:
        st_ = (c_ll * len(steps))(*steps)
        tg = (c_double * len(steps))(*p.sample_targets)
        wt = (c_double * len(steps))(*p.sample_weights)
        keep += [st_, tg, wt]
        s.sample_step = ctypes.cast(st_, ctypes.POINTER(c_ll))
        s.sample_target = ctypes.cast(tg, _PD)
        s.sample_weight = ctypes.cast(wt, _PD)
    s.nsample = len(steps)
    s.centre_w = getattr(p, "centre_w", 0.0)
    s.centre_target[:] = list(getattr(p, "centre_target", (0.0, 0.0)))
    s._keep = keep
    return s


def _check(lib, ctx, st):
    if st != LLG_OK:
        msg = lib.llg_last_error(ctx)
        raise LLGError(st, msg.decode() if msg else "")


# ---- thin wrappers with the C names -------------------------------------

def llg_create(problems: Sequence, precision=LLG_FP32, ckpt=LLG_CKPT_PERIODIC, seg_len=0,
               stream=0, tune=LLG_TUNE_DEFAULT, use_graph=0, time_kernels=0,
               integrator=LLG_INT_RK4, rtol=1e-6, atol=1e-9, adj_spectral=LLG_SPEC_WORKING,
               launch=None, record=LLG_RECORD_STAGES) -> int:
    lib = load()
    structs = [to_struct(p) for p in problems]          # hold the host arrays until create returns
    arr = (llg_problem * len(problems))(*structs)
    lc = llg_launch(**launch) if launch else llg_launch(16, 2, 2, 2, 1)
    opt = llg_options(precision, ckpt, seg_len, use_graph, tune, time_kernels, integrator,
                      rtol, atol, adj_spectral, lc, record)
    ctx = c_void_p()
    st = lib.llg_create(arr, len(problems), ctypes.byref(opt), c_void_p(stream), ctypes.byref(ctx))
    if st != LLG_OK:
        msg = lib.llg_last_error(ctx).decode() if ctx.value else ""
        if ctx.value:
            lib.llg_destroy(ctx)
        raise LLGError(st, msg)
    return ctx.value


def llg_forward(ctx: int, phi_ptr: int, m0_ptr: int, n_inst: int, mT_ptr: int = 0) -> np.ndarray:
    lib = load()
    J = (c_double * n_inst)()
    _check(lib, ctx, lib.llg_forward(c_void_p(ctx), c_void_p(phi_ptr), c_void_p(m0_ptr), J,
                                     c_void_p(mT_ptr or None)))
    return np.array(J[:])


def llg_adjoint(ctx: int, dphi_ptr: int, dm0_ptr: int = 0, dJ_dextra=None) -> None:
    """dJ_dextra: optional per-instance cotangents of J (host sequence)."""
    lib = load()
    w = None if dJ_dextra is None else (c_double * len(dJ_dextra))(*[float(v) for v in dJ_dextra])
    _check(lib, ctx, lib.llg_adjoint(c_void_p(ctx), w, c_void_p(dphi_ptr), c_void_p(dm0_ptr or None)))


def llg_launch_config(ctx: int):
    """(launch configuration as a dict, ms spent timing candidates at create)."""
    lib = load()
    out = llg_launch()
    ms = c_double()
    _check(lib, ctx, lib.llg_launch_config(c_void_p(ctx), ctypes.byref(out), ctypes.byref(ms)))
    return out.as_dict(), ms.value


def levelset_step(ctx: int, phi_ptr: int, grad_ptr: int, mask_ptr: int, lr: float) -> None:
    lib = load()
    _check(lib, ctx, lib.levelset_step(c_void_p(ctx), c_void_p(phi_ptr), c_void_p(grad_ptr),
                                       c_void_p(mask_ptr), lr))


def llg_field(ctx: int, phi_ptr: int, m_ptr: int, t: float, demag_only: bool, B_ptr: int) -> None:
    lib = load()
    _check(lib, ctx, lib.llg_field(c_void_p(ctx), c_void_p(phi_ptr), c_void_p(m_ptr), t,
                                   int(bool(demag_only)), c_void_p(B_ptr)))


def llg_field_noalloc(problem, phi_ptr: int, m_ptr: int, t: float, demag_only: bool, B_ptr: int,
                      stream: int = 0) -> None:
    """Field of one FP32 instance with the library's fixed scratch (no device
    allocation; grids up to 128 x 128).  Queued on `stream`."""
    lib = load()
    s = to_struct(problem)
    msg = ctypes.c_char_p()
    st = lib.llg_field_noalloc(ctypes.byref(s), c_void_p(phi_ptr), c_void_p(m_ptr), t, int(bool(demag_only)),
                               c_void_p(B_ptr), c_void_p(stream), ctypes.byref(msg))
    if st != LLG_OK:
        raise LLGError(st, msg.value.decode() if msg.value else "")


def make_rbf(nx: int, ny: int, dx: float, dy: float, box, nrx: int, nry: int, p: float = 90.0) -> llg_rbf:
    return llg_rbf(nx, ny, dx, dy, (c_int * 4)(*box), nrx, nry, p)


def llg_rbf_workspace_bytes(r: llg_rbf) -> int:
    return int(load().llg_rbf_workspace_bytes(ctypes.byref(r)))


def _rbf_check(st: int, what: str) -> None:
    if st != LLG_OK:
        raise LLGError(st, f"{what}: invalid arguments" if st == LLG_EINVAL else f"{what}: CUDA launch failed")


def llg_rbf_phi(r: llg_rbf, s_ptr: int, phi_ptr: int, precision: int, work_ptr: int, stream: int = 0) -> None:
    """Phi on the design box from the RBF amplitudes (Eq. 2, 3, renormalised)."""
    _rbf_check(load().llg_rbf_phi(ctypes.byref(r), c_void_p(s_ptr), c_void_p(phi_ptr), precision,
                                  c_void_p(work_ptr), c_void_p(stream)), "llg_rbf_phi")


def llg_rbf_grad(r: llg_rbf, s_ptr: int, dJdphi_ptr: int, precision: int, dJds_ptr: int, work_ptr: int,
                 stream: int = 0) -> None:
    """dJ/ds from dJ/dPhi through the RBF map."""
    _rbf_check(load().llg_rbf_grad(ctypes.byref(r), c_void_p(s_ptr), c_void_p(dJdphi_ptr), precision,
                                   c_void_p(dJds_ptr), c_void_p(work_ptr), c_void_p(stream)), "llg_rbf_grad")


def llg_adam_step(s_ptr: int, grad_ptr: int, m_ptr: int, v_ptr: int, n: int, t: int, lr: float,
                  b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8, stream: int = 0) -> None:
    """One Adam step on n double parameters (step number t >= 1)."""
    _rbf_check(load().llg_adam_step(c_void_p(s_ptr), c_void_p(grad_ptr), c_void_p(m_ptr), c_void_p(v_ptr), n, t,
                                    lr, b1, b2, eps, c_void_p(stream)), "llg_adam_step")


def llg_fp64_fma_rate(iters: int = 16384, stream: int = 0):
    """Measured FP64 FMA throughput of the current device: (TFLOP/s, ms of
    the best launch)."""
    tf, ms = c_double(), c_double()
    _rbf_check(load().llg_fp64_fma_rate(iters, ctypes.byref(tf), ctypes.byref(ms), c_void_p(stream)),
               "llg_fp64_fma_rate")
    return tf.value, ms.value


def llg_adaptive_steps(ctx: int, inst: int):
    """Accepted steps (t_k, h_k) of instance `inst` in the last adaptive
    forward pass, as two numpy arrays."""
    lib = load()
    count = c_ll()
    _check(lib, ctx, lib.llg_adaptive_steps(c_void_p(ctx), inst, None, None, 0, ctypes.byref(count)))
    K = count.value
    t = (c_double * max(1, K))()
    h = (c_double * max(1, K))()
    _check(lib, ctx, lib.llg_adaptive_steps(c_void_p(ctx), inst, t, h, K, ctypes.byref(count)))
    return np.array(t[:K]), np.array(h[:K])


def llg_query(ctx: int):
    lib = load()
    b = ctypes.c_size_t()
    ms = c_double()
    _check(lib, ctx, lib.llg_query(c_void_p(ctx), ctypes.byref(b), ctypes.byref(ms)))
    return b.value, ms.value


def llg_launch_count(ctx: int) -> int:
    return load().llg_launch_count(c_void_p(ctx))


def llg_kernel_time(ctx: int, family: int):
    """(launches, total_ms) of a kernel family: 0 row stage, 1 column, 2 adjoint,
    3 column pass of the double-float adjoint spectrum, 4 its row transforms
    (split adjoint stage)."""
    lib = load()
    n = c_ll()
    ms = c_double()
    _check(lib, ctx, lib.llg_kernel_time(c_void_p(ctx), family, ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def llg_last_error(ctx: int) -> str:
    return load().llg_last_error(c_void_p(ctx)).decode()


def llg_destroy(ctx: int) -> None:
    load().llg_destroy(c_void_p(ctx))


def llg_schedule(nsteps: int, ckpt: int = LLG_CKPT_PERIODIC, seg_len: int = 0):
    """(forward_actions, reverse_actions) as lists of (op, a, b)."""
    lib = load()
    nf = c_ll()
    tot = lib.llg_schedule(nsteps, ckpt, seg_len, None, 0, ctypes.byref(nf))
    if tot < 0:
        raise LLGError(LLG_EINVAL, "bad schedule arguments")
    buf = (c_ll * (3 * max(tot, 1)))()
    lib.llg_schedule(nsteps, ckpt, seg_len, buf, tot, ctypes.byref(nf))
    acts = [tuple(buf[3 * k:3 * k + 3]) for k in range(tot)]
    return acts[:nf.value], acts[nf.value:]


def llg_padded_extents(nx: int, ny: int):
    px, py = c_int(), c_int()
    load().llg_padded_extents(nx, ny, ctypes.byref(px), ctypes.byref(py))
    return px.value, py.value


# ---- torch convenience layer ------------------------------------------------

class Solver:
    """A batch of instances on one GPU.  Inputs and outputs are torch CUDA
    tensors packed back to back in instance order (phi: [sum n_i], m:
    [sum 3 n_i] with each instance laid out [3][ny][nx])."""

    def __init__(self, problems: Sequence, precision: str = "fp32", ckpt: str = "periodic",
                 seg_len: int = 0, stream=None, tune: str = "default", launch=None,
                 time_kernels: bool = False, use_graph: bool = True, integrator: str = "rk4",
                 rtol: float = 1e-6, atol: float = 1e-9, adj_spectral: str = "working", record: str = "stages"):
        """tune: "default", "measure" (time launch candidates at create) or
        "given" (use `launch`, a dict of llg_launch fields)."""
        import torch
        self.torch = torch
        self.problems = list(problems)
        self.dtype = torch.float32 if precision == "fp32" else torch.float64
        prec = LLG_FP32 if precision == "fp32" else LLG_FP64
        ck = {"periodic": LLG_CKPT_PERIODIC, "store_all": LLG_CKPT_STORE_ALL, "binomial": LLG_CKPT_BINOMIAL}[ckpt]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        integ = {"rk4": LLG_INT_RK4, "dopri5": LLG_INT_DOPRI5}[integrator]
        spec = {"working": LLG_SPEC_WORKING, "dfloat": LLG_SPEC_DFLOAT}[adj_spectral]
        tn = {"default": LLG_TUNE_DEFAULT, "measure": LLG_TUNE_MEASURE, "given": LLG_TUNE_GIVEN}[tune]
        self.ctx = llg_create(self.problems, prec, ck, seg_len, self.stream.cuda_stream,
                              tn, int(use_graph), int(time_kernels), integ, rtol, atol, spec, launch,
                              {"stages": LLG_RECORD_STAGES, "states": LLG_RECORD_STATES}[record])
        self.nodes = [p.nx * p.ny * p.nz for p in self.problems]
        self.total = sum(self.nodes)

    def close(self):
        if getattr(self, "ctx", None):
            llg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # packing helpers ---------------------------------------------------
    def pack_scalar(self, arrays) -> "torch.Tensor":
        t = self.torch
        return t.cat([t.as_tensor(np.asarray(a).reshape(-1), dtype=self.dtype) for a in arrays]).cuda()

    def pack_vector(self, arrays) -> "torch.Tensor":
        return self.pack_scalar(arrays)

    def unpack_scalar(self, x):
        out, o = [], 0
        for p, k in zip(self.problems, self.nodes):
            out.append(x[o:o + k].reshape(p.nz, p.ny, p.nx))
            o += k
        return out

    def unpack_vector(self, x):
        out, o = [], 0
        for p, k in zip(self.problems, self.nodes):
            out.append(x[o:o + 3 * k].reshape(3, p.nz, p.ny, p.nx))
            o += 3 * k
        return out

    def _chk(self, x, n):
        t = self.torch
        if not (isinstance(x, t.Tensor) and x.is_cuda and x.dtype == self.dtype and x.is_contiguous()
                and x.numel() == n):
            raise ValueError(f"expected a contiguous CUDA {self.dtype} tensor with {n} elements")
        return x.data_ptr()

    # calls ---------------------------------------------------------------
    def forward(self, phi, m0, want_mT: bool = False):
        mT = self.torch.empty(3 * self.total, dtype=self.dtype, device="cuda") if want_mT else None
        J = llg_forward(self.ctx, self._chk(phi, self.total), self._chk(m0, 3 * self.total),
                        len(self.problems), mT.data_ptr() if mT is not None else 0)
        return J, mT

    def adjoint(self, want_dm0: bool = False, dJ_dextra=None):
        """dJ/dPhi (and dJ/dm0) of sum_i dJ_dextra[i] J_i (all ones if None)."""
        g = self.torch.empty(self.total, dtype=self.dtype, device="cuda")
        dm0 = self.torch.empty(3 * self.total, dtype=self.dtype, device="cuda") if want_dm0 else None
        llg_adjoint(self.ctx, g.data_ptr(), dm0.data_ptr() if dm0 is not None else 0, dJ_dextra)
        return g, dm0

    def launch_config(self):
        return llg_launch_config(self.ctx)

    def levelset_step(self, phi, grad, mask, lr: float):
        if mask.dtype != self.torch.uint8 or not mask.is_cuda:
            raise ValueError("mask must be a CUDA uint8 tensor")
        levelset_step(self.ctx, self._chk(phi, self.total), self._chk(grad, self.total), mask.data_ptr(), lr)
        return phi

    def field(self, phi, m, t: float = 0.0, demag_only: bool = False):
        B = self.torch.empty(3 * self.total, dtype=self.dtype, device="cuda")
        llg_field(self.ctx, self._chk(phi, self.total), self._chk(m, 3 * self.total), t, demag_only,
                  B.data_ptr())
        return B

    def query(self):
        return llg_query(self.ctx)

    def launch_count(self) -> int:
        return llg_launch_count(self.ctx)

    def adaptive_steps(self, inst: int):
        """(t_k, h_k) of the accepted steps of instance `inst` (dopri5)."""
        return llg_adaptive_steps(self.ctx, inst)

    def kernel_time(self, family: int):
        return llg_kernel_time(self.ctx, family)


def _make_function():
    import torch

    class LLGFunction(torch.autograd.Function):
        """J = LLGFunction.apply(phi, m0, solver): forward pass of the solver;
        backward runs the hand-written adjoint sweep (no autograd tape)."""

        @staticmethod
        def forward(ctx, phi, m0, solver):
            J, _ = solver.forward(phi.contiguous(), m0.contiguous())
            ctx.solver = solver
            ctx.counts = solver.nodes
            return torch.as_tensor(J, dtype=torch.float64, device=phi.device)

        @staticmethod
        def backward(ctx, gJ):
            # the incoming cotangents of the instances' J seed the adjoint
            g, dm0 = ctx.solver.adjoint(want_dm0=True, dJ_dextra=gJ.double().cpu().tolist())
            return g, dm0, None

    return LLGFunction


_fn = None


def llg_function():
    global _fn
    if _fn is None:
        _fn = _make_function()
    return _fn
