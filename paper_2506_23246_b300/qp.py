"""Thin ctypes binding of libqpinn.so (C-ABI declared in include/qpinn.h).

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels. PyTorch provides device memory and streams. There is no fallback: if the
extension is missing or fails to load, every call raises.
"""
import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqpinn.so")

ANSATZ = {"basic_ryrz": 0, "basic_rot": 1, "strong_rot": 2, "noent_rot": 3, "cross_mesh": 4,
          "cross_mesh_2rot": 5, "cross_mesh_cnot": 6}
ENC = {"rx": 0, "ry": 1}
SCALE = {"none": 0, "pi": 1, "bias": 2, "asin": 3, "acos": 4}
PREMAP = {"direct": 0, "rff_mlp": 1}
PATH = {"auto": 0, "simt": 1, "gemm_split": 2, "gemm_bf16x3": 3}
OPERANDS = {"fp16_pairs": 0, "tf32_pairs": 1}
NLOSS = 9
PHYS_LOSS = {"split": 0, "intuitive": 1}
STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported configuration",
          3: "workspace missing or too small", 4: "CUDA error", 5: "non-finite loss",
          6: "device wait timed out", 7: "internal error"}


class QPError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s: %s (status %d)" % (what, STATUS.get(code, "?"), code))
        self.code = code


class QPCircuit(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in (
        "n_qubits", "n_layers", "n_readout", "ansatz", "enc", "scale", "premap", "n_direct",
        "rff_freqs", "mlp_width", "mlp_depth", "periodic")]


class QPProblem(ctypes.Structure):
    _fields_ = [("medium", ctypes.c_int32)] + [(k, ctypes.c_float) for k in (
        "eps_r", "disk_r", "disk_x0", "disk_y0", "sigmoid_w", "ic_sigma", "ic_x0", "ic_y0",
        "w_ic", "w_bc", "w_energy")] + [("energy_slice", ctypes.c_int32),
                                        ("energy_nt", ctypes.c_int32),
                                        ("phys_loss", ctypes.c_int32), ("w_sym", ctypes.c_float)]


class QPBatch(ctypes.Structure):
    _fields_ = [("colloc", ctypes.c_void_p), ("n_colloc", ctypes.c_int64),
                ("ic", ctypes.c_void_p), ("n_ic", ctypes.c_int64),
                ("bc", ctypes.c_void_p), ("n_bc", ctypes.c_int64),
                ("norm_colloc", ctypes.c_int64), ("norm_ic", ctypes.c_int64),
                ("norm_bc", ctypes.c_int64), ("norm_diel", ctypes.c_int64),
                ("colloc_offset", ctypes.c_int64)]


class QPStepArgs(ctypes.Structure):
    _fields_ = [("d_params", ctypes.c_void_p), ("batch", QPBatch), ("d_loss", ctypes.c_void_p),
                ("d_grad", ctypes.c_void_p)]


_lib = None


def lib():
    """Load libqpinn.so (raises if it is missing: there is no other implementation)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libqpinn.so not built: run python -m paper_2506_23246_b300.build")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.qp_plan_create.argtypes = [ctypes.POINTER(QPCircuit), ctypes.POINTER(QPProblem), I32,
                                     ctypes.POINTER(P)]
        L.qp_plan_create.restype = I32
        L.qp_plan_destroy.argtypes = [P]
        L.qp_plan_destroy.restype = None
        L.qp_param_count.argtypes = [P, ctypes.POINTER(I64)]
        L.qp_param_layout.argtypes = [P, ctypes.POINTER(I64)]
        L.qp_workspace_size.argtypes = [P, I64, ctypes.POINTER(ctypes.c_size_t)]
        L.qp_set_workspace.argtypes = [P, P, ctypes.c_size_t]
        L.qp_forward.argtypes = [P, P, P, I64, P, P, P]
        L.qp_loss_grad.argtypes = [P, P, ctypes.POINTER(QPBatch), P, P, P]
        L.qp_count_dielectric.argtypes = [P, P, I64, P, P]
        L.qp_batch_step.argtypes = [ctypes.POINTER(P), I32, ctypes.POINTER(QPStepArgs), P]
        L.qp_batch_step_flags.argtypes = [ctypes.POINTER(P), I32, ctypes.POINTER(QPStepArgs), P, ctypes.c_uint32]
        L.qp_batch_tune.argtypes = [ctypes.POINTER(P), I32, ctypes.POINTER(QPStepArgs), P, ctypes.POINTER(I32)]
        L.qp_last_device_error.argtypes = [P]
        L.qp_status_str.argtypes = [I32]
        L.qp_status_str.restype = ctypes.c_char_p
        L.qp_last_launch_count.argtypes = [P]
        L.qp_last_launch_count.restype = I32
        L.qp_plan_path.argtypes = [P]
        L.qp_plan_path.restype = I32
        L.qp_plan_set_operands.argtypes = [P, I32]
        L.qp_plan_set_operands.restype = I32
        L.qp_bh_indicator.argtypes = [P, I32, ctypes.c_double, ctypes.c_double, P, P]
        L.qp_bh_indicator.restype = I32
        L.qp_set_wait_limit.argtypes = [P, ctypes.c_uint32]
        L.qp_set_wait_limit.restype = I32
        L.qp_set_profile_events.argtypes = [P, I32, P, P]
        L.qp_set_profile_events.restype = I32
        L.qp_sched_selftest.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint]
        L.qp_sched_selftest.restype = ctypes.c_double
        L.qp_sched_conflicts.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.qp_sched_conflicts.restype = ctypes.c_int
        for name in ("qp_param_count", "qp_param_layout", "qp_workspace_size", "qp_set_workspace",
                     "qp_forward", "qp_loss_grad", "qp_last_device_error"):
            getattr(L, name).restype = I32
        _lib = L
    return _lib


def _check(code, what):
    if code != 0:
        raise QPError(code, what)


def make_circuit(c):
    return QPCircuit(c["n_qubits"], c["n_layers"], c["n_readout"], ANSATZ[c["ansatz"]],
                     ENC[c["enc"]], SCALE[c["scale"]], PREMAP[c["premap"]], c.get("n_direct", 3),
                     c.get("rff_freqs", 0), c.get("mlp_width", 0), c.get("mlp_depth", 0),
                     1 if c.get("periodic") else 0)


def make_problem(p):
    return QPProblem(1 if p["medium"] == "dielectric" else 0, p["eps_r"], p["disk_r"],
                     p["disk_x0"], p["disk_y0"], p["sigmoid_w"], p["ic_sigma"], p["ic_x0"],
                     p["ic_y0"], p["w_ic"], p["w_bc"], p["w_energy"], p.get("energy_slice", 0),
                     p.get("energy_nt", 0), PHYS_LOSS[p.get("phys_loss", "split")],
                     float(p.get("w_sym", 0.0)))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _dev_f32(t, device, what):
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise ValueError("%s must be a CUDA tensor" % what)
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("%s must be contiguous float32" % what)
    return t


class Plan:
    """One circuit + problem configuration (qp_plan) with its device workspace."""

    def __init__(self, circuit, problem=None, path="auto", operands="fp16_pairs"):
        from . import workloads
        self.circuit = dict(circuit)
        self.problem = dict(problem or workloads.problem())
        self._c = make_circuit(self.circuit)
        self._p = make_problem(self.problem)
        h = ctypes.c_void_p()
        _check(lib().qp_plan_create(ctypes.byref(self._c), ctypes.byref(self._p), PATH[path],
                                    ctypes.byref(h)), "qp_plan_create")
        self._h = h
        self._ws = None
        self._ws_points = -1
        n = ctypes.c_int64()
        _check(lib().qp_param_count(self._h, ctypes.byref(n)), "qp_param_count")
        self.n_params = n.value
        lay = (ctypes.c_int64 * 4)()
        _check(lib().qp_param_layout(self._h, lay), "qp_param_layout")
        self.layout = {"circuit": lay[0], "head": lay[1], "total": lay[2], "fixed": lay[3]}
        self.path = {1: "simt", 2: "gemm_split"}.get(lib().qp_plan_path(self._h), "?")
        _check(lib().qp_plan_set_operands(self._h, OPERANDS[operands]), "qp_plan_set_operands")
        self.operands = operands

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.qp_plan_destroy(h)
            self._h = None

    def workspace_bytes(self, npoints):
        b = ctypes.c_size_t()
        _check(lib().qp_workspace_size(self._h, int(npoints), ctypes.byref(b)), "qp_workspace_size")
        return b.value

    def reserve(self, npoints, device="cuda"):
        """Allocate (through torch) and attach a workspace for up to npoints points."""
        if npoints <= self._ws_points and self._ws is not None:
            return
        nbytes = self.workspace_bytes(npoints)
        self._ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
        _check(lib().qp_set_workspace(self._h, _ptr(self._ws), self._ws.numel()), "qp_set_workspace")
        self._ws_points = npoints

    @staticmethod
    def _stream(stream):
        s = stream if stream is not None else torch.cuda.current_stream()
        return ctypes.c_void_p(s.cuda_stream)

    def forward(self, params, pts, want_df=True, out=None, stream=None):
        """Fields [B,3] and (optionally) input derivatives [B,3,3] at pts [B,3]."""
        _dev_f32(params, None, "params")
        _dev_f32(pts, None, "pts")
        B = pts.shape[0]
        self.reserve(B, pts.device)
        if out is None:
            f = torch.empty(B, 3, dtype=torch.float32, device=pts.device)
            df = torch.empty(B, 3, 3, dtype=torch.float32, device=pts.device) if want_df else None
        else:
            f, df = out
        _check(lib().qp_forward(self._h, _ptr(params), _ptr(pts), B, _ptr(f), _ptr(df),
                                self._stream(stream)), "qp_forward")
        return f, df

    def _batch(self, params, sets, norm):
        _dev_f32(params, None, "params")
        if params.numel() != self.n_params:
            raise ValueError("params has %d entries, plan expects %d" % (params.numel(), self.n_params))
        ts = {}
        for k in ("colloc", "ic", "bc"):
            t = sets.get(k)
            if t is not None and t.shape[0] > 0:
                ts[k] = _dev_f32(t, None, k)
        total = sum(t.shape[0] for t in ts.values())
        self.reserve(total, params.device)
        nm = norm or {}
        batch = QPBatch(
            _ptr(ts.get("colloc")), ts["colloc"].shape[0] if "colloc" in ts else 0,
            _ptr(ts.get("ic")), ts["ic"].shape[0] if "ic" in ts else 0,
            _ptr(ts.get("bc")), ts["bc"].shape[0] if "bc" in ts else 0,
            int(nm.get("n_colloc", 0)), int(nm.get("n_ic", 0)), int(nm.get("n_bc", 0)),
            int(nm.get("n_diel", 0)), int(nm.get("colloc_offset", 0)))
        return batch, ts

    def _outputs(self, params, out):
        if out is not None:
            return out
        nl = NLOSS + self.problem.get("energy_nt", 0) + (1 if self.problem.get("w_sym", 0.0) > 0 else 0)
        return (torch.empty(nl, dtype=torch.float64, device=params.device),
                torch.empty(self.n_params, dtype=torch.float32, device=params.device))

    def loss_grad(self, params, sets, out=None, stream=None, norm=None):
        """Loss terms (float64 [9 + energy_nt]) and d total / d params (float32 [n_params]).
        norm: sharding of one loss over several calls (dict: whole-loss counts n_colloc, n_ic,
        n_bc, whole-set n_diel, colloc_offset); see qp_batch in qpinn.h."""
        batch, _ = self._batch(params, sets, norm)
        loss, grad = self._outputs(params, out)
        _check(lib().qp_loss_grad(self._h, _ptr(params), ctypes.byref(batch), _ptr(loss), _ptr(grad),
                                  self._stream(stream)), "qp_loss_grad")
        return loss, grad

    def count_dielectric(self, pts, out=None, stream=None):
        """Number of points of pts [n,3] inside the dielectric disk, as a device int64 [1]."""
        n = pts.shape[0]
        if n > 0:
            _dev_f32(pts, None, "pts")
        c = out if out is not None else torch.empty(1, dtype=torch.int64, device=pts.device)
        _check(lib().qp_count_dielectric(self._h, _ptr(pts) if n > 0 else None, n, _ptr(c),
                                         self._stream(stream)), "qp_count_dielectric")
        return c

    def last_device_error(self):
        return lib().qp_last_device_error(self._h)

    def set_wait_limit(self, polls):
        """Test hook: bound the fused forward's pipeline waits to `polls` polls (0: default)."""
        _check(lib().qp_set_wait_limit(self._h, int(polls)), "qp_set_wait_limit")

    def last_launch_count(self):
        return lib().qp_last_launch_count(self._h)

    PROF = {"main": 0, "wgrad": 1, "mu": 2}

    def set_profile_events(self, start=None, stop=None, kernel="main"):
        """Record two torch.cuda.Event objects around one measured kernel of later calls:
        "main" (the statevector kernel, or the forward contraction on the tensor-core path),
        "wgrad" (weight-gradient contraction) or "mu" (back-projection)."""
        if start is not None:
            # torch creates the CUDA event on first record; make sure both handles exist
            start.record()
            stop.record()
            torch.cuda.synchronize()
        s = ctypes.c_void_p(start.cuda_event) if start is not None else ctypes.c_void_p(0)
        e = ctypes.c_void_p(stop.cuda_event) if stop is not None else ctypes.c_void_p(0)
        _check(lib().qp_set_profile_events(self._h, self.PROF[kernel], s, e), "qp_set_profile_events")


def bh_indicator(loss_terms, energy_nt, t_max, delta, out=None, stream=None):
    """Black-hole collapse indicator (Sec. 5) from the loss terms of loss_grad: a float64
    device tensor [energy_nt + 1], the normalised energies U(t_k) / U(0) then I_BH."""
    if not isinstance(loss_terms, torch.Tensor) or loss_terms.device.type != "cuda" or \
            loss_terms.dtype != torch.float64 or not loss_terms.is_contiguous():
        raise ValueError("loss_terms must be a contiguous float64 CUDA tensor")
    if loss_terms.numel() < NLOSS + energy_nt:
        raise ValueError("loss_terms holds fewer than 9 + energy_nt values")
    if out is None:
        out = torch.empty(energy_nt + 1, dtype=torch.float64, device=loss_terms.device)
    s = stream if stream is not None else torch.cuda.current_stream(loss_terms.device)
    _check(lib().qp_bh_indicator(_ptr(loss_terms), int(energy_nt), float(t_max), float(delta), _ptr(out),
                                 ctypes.c_void_p(s.cuda_stream)), "qp_bh_indicator")
    return out


BATCH_NO_GROUPING = 1


def _step_args(plans, params, sets, outs, norms):
    k = len(plans)
    outs = outs or [None] * k
    norms = norms or [None] * k
    arr = (QPStepArgs * max(k, 1))()
    handles = (ctypes.c_void_p * max(k, 1))()
    keep, res = [], []
    for i in range(k):
        batch, ts = plans[i]._batch(params[i], sets[i], norms[i])
        loss, grad = plans[i]._outputs(params[i], outs[i])
        keep.append(ts)
        arr[i] = QPStepArgs(_ptr(params[i]), batch, _ptr(loss), _ptr(grad))
        handles[i] = plans[i]._h
        res.append((loss, grad))
    return handles, arr, keep, res


def batch_step(plans, params, sets, outs=None, norms=None, stream=None, grouped=True):
    """Loss and gradient of independent instances in one qp_batch_step call: plans[i] with
    params[i] on sets[i]; returns [(loss, grad)] in the order given. grouped=False: every
    instance as its own call on the worker streams (no multi-instance launch)."""
    handles, arr, keep, res = _step_args(plans, params, sets, outs, norms)
    s = stream if stream is not None else torch.cuda.current_stream()
    flags = 0 if grouped else BATCH_NO_GROUPING
    _check(lib().qp_batch_step_flags(handles, len(plans), arr, ctypes.c_void_p(s.cuda_stream), flags),
           "qp_batch_step_flags")
    return res


def batch_tune(plans, params, sets, outs=None, norms=None, stream=None):
    """Time the multi-instance launch shapes on this mix and keep the fastest in its plans
    (qp_batch_tune); returns (warps per CTA, tasks per warp and item)."""
    handles, arr, keep, res = _step_args(plans, params, sets, outs, norms)
    s = stream if stream is not None else torch.cuda.current_stream()
    ch = (ctypes.c_int32 * 2)()
    _check(lib().qp_batch_tune(handles, len(plans), arr, ctypes.c_void_p(s.cuda_stream), ch), "qp_batch_tune")
    return int(ch[0]), int(ch[1])


class QPINNLoss(torch.autograd.Function):
    """Total loss (Eq. 24 without L_sym) as a differentiable function of the flat parameter
    vector; the backward pass returns the gradient the library's adjoint sweep computed."""

    @staticmethod
    def forward(ctx, params, plan, sets):
        loss, grad = plan.loss_grad(params.detach().contiguous(), sets)
        ctx.save_for_backward(grad)
        ctx.mark_non_differentiable(loss)
        return loss[0].to(params.dtype), loss

    @staticmethod
    def backward(ctx, g_total, g_terms):
        (grad,) = ctx.saved_tensors
        return grad * g_total, None, None


def qpinn_loss(params, plan, sets):
    total, terms = QPINNLoss.apply(params, plan, sets)
    return total, terms
