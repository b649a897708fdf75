"""Thin ctypes binding of libsgpe (include/sgpe.h): argument marshalling only.

Every substep of the method runs in the library's CUDA kernels; PyTorch only
provides device memory (state, workspace) and the CUDA stream. There is no CPU
fallback: if the library has not been built, loading it raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, asdict

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsgpe.so")
_lib = None

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, ESTATE, EUNSUPPORTED = range(8)
STATUS = {0: "SGPE_OK", 1: "SGPE_EINVAL", 2: "SGPE_ENOMEM", 3: "SGPE_ECUDA", 4: "SGPE_ENONFINITE",
          5: "SGPE_ETIMEOUT", 6: "SGPE_ESTATE", 7: "SGPE_EUNSUPPORTED"}
C128, C64, CDF = 0, 1, 2
PRECISIONS = {"c128": C128, "c64": C64, "cdf": CDF}
NOBS = 16
OBS_NAMES = ("N+", "N0", "N-", "N", "mag", "E", "mu", "rms+", "rms0", "rms-", "rms",
             "E_kin", "E_trap", "E_int", "E_rabi", "E_so")
SUBSTEP = {"so": 0, "calcnu": 1, "herm": 2, "cn_x": 3, "cn_y": 4, "renorm": 5, "so_cn": 6, "so_cn_rev": 7}

# Every symbol include/sgpe.h declares (checked by the CPU test suite).
EXPORTS = ("sgpe_init_grid", "sgpe_workspace_bytes", "sgpe_bind", "sgpe_set_params", "sgpe_step_imag",
           "sgpe_step_real", "sgpe_normalize", "sgpe_energy", "sgpe_set_state", "sgpe_get_state", "sgpe_load_state",
           "sgpe_substep", "sgpe_profile_steps", "sgpe_measure_fp64_rate", "sgpe_eval_expm1f",
           "sgpe_observables_noalloc", "sgpe_launches_per_step",
           "sgpe_last_error", "sgpe_destroy", "sgpe_adjoint_workspace_bytes", "sgpe_adjoint_loss_grad",
           "sgpe_adjoint_forward", "sgpe_adjoint_step",
           "sgpe_batch_create", "sgpe_batch_sizes", "sgpe_batch_offsets", "sgpe_batch_bind",
           "sgpe_batch_load_state", "sgpe_batch_step_imag", "sgpe_batch_step_real", "sgpe_batch_energy",
           "sgpe_batch_autotune", "sgpe_batch_set_tiles", "sgpe_batch_launches_per_step", "sgpe_batch_last_error",
           "sgpe_batch_destroy")


class SgpeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class Params(ctypes.Structure):
    """sgpe_params (include/sgpe.h)."""
    _fields_ = [("c0", ctypes.c_double), ("c2", ctypes.c_double), ("so_type", ctypes.c_int),
                ("gamma", ctypes.c_double), ("omega", ctypes.c_double), ("wx", ctypes.c_double),
                ("wy", ctypes.c_double), ("dt", ctypes.c_double), ("renorm", ctypes.c_int),
                ("mag", ctypes.c_double), ("split", ctypes.c_int), ("so_mode", ctypes.c_int)]


def load():
    """Load libsgpe.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libsgpe.so not found at %s; build it first (python -c 'import __graft_entry__ as g; "
                           "g.build()')" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sig = {
        "sgpe_init_grid": (I, [ctypes.POINTER(P), I, I, I, D, D, I, P]),
        "sgpe_workspace_bytes": (I, [P, ctypes.POINTER(S)]),
        "sgpe_bind": (I, [P, P, P]),
        "sgpe_set_params": (I, [P, ctypes.POINTER(Params)]),
        "sgpe_step_imag": (I, [P, I]),
        "sgpe_step_real": (I, [P, I, P]),
        "sgpe_normalize": (I, [P, P]),
        "sgpe_energy": (I, [P, P]),
        "sgpe_set_state": (I, [P, P]),
        "sgpe_get_state": (I, [P, P]),
        "sgpe_load_state": (I, [P, P]),
        "sgpe_substep": (I, [P, I, I, D]),
        "sgpe_profile_steps": (I, [P, I, I, P, P]),
        "sgpe_measure_fp64_rate": (I, [P, P]),
        "sgpe_eval_expm1f": (I, [P, P, P, I]),
        "sgpe_observables_noalloc": (I, [P, I, I, I, D, D, I, ctypes.POINTER(Params), P, P]),
        "sgpe_launches_per_step": (I, [P]),
        "sgpe_last_error": (ctypes.c_char_p, [P]),
        "sgpe_destroy": (I, [P]),
        "sgpe_adjoint_workspace_bytes": (I, [P, I, I, ctypes.POINTER(S)]),
        "sgpe_adjoint_loss_grad": (I, [P, I, P, P, I, P, P, P, P]),
        "sgpe_adjoint_forward": (I, [P, I, P, I, P]),
        "sgpe_adjoint_step": (I, [P, I, P, I, P, P, P, P]),
        "sgpe_batch_create": (I, [ctypes.POINTER(P), I, P, I, P]),
        "sgpe_batch_sizes": (I, [P, ctypes.POINTER(S), ctypes.POINTER(S)]),
        "sgpe_batch_offsets": (I, [P, P]),
        "sgpe_batch_bind": (I, [P, P, P]),
        "sgpe_batch_load_state": (I, [P, P]),
        "sgpe_batch_step_imag": (I, [P, I]),
        "sgpe_batch_step_real": (I, [P, I]),
        "sgpe_batch_energy": (I, [P, P]),
        "sgpe_batch_autotune": (I, [P, I, P]),
        "sgpe_batch_set_tiles": (I, [P, I, I]),
        "sgpe_batch_launches_per_step": (I, [P]),
        "sgpe_batch_last_error": (ctypes.c_char_p, [P]),
        "sgpe_batch_destroy": (I, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


@dataclass
class Physics:
    """Physical parameters (sgpe_params)."""
    c0: float = 0.0
    c2: float = 0.0
    so_type: int = 0
    gamma: float = 0.0
    omega: float = 0.0
    wx: float = 1.0
    wy: float = 1.0
    dt: float = 1e-4
    renorm: int = 1
    mag: float = 0.0
    split: int = 0      # 0 Lie, 1 Strang splitting
    so_mode: int = 0    # 0 explicit-Euler SO, 1 SO by Crank-Nicolson (unitary)

    def c(self) -> Params:
        return Params(self.c0, self.c2, self.so_type, self.gamma, self.omega, self.wx, self.wy, self.dt,
                      self.renorm, self.mag, self.split, self.so_mode)


class Solver:
    """One grid on one GPU: state and workspace are torch tensors, the step runs in libsgpe."""

    def __init__(self, dim, nx, ny=1, dx=0.05, dy=None, precision="c128", device="cuda:0", stream=None):
        import torch
        self.torch = torch
        self.lib = load()
        self.dim, self.nx = int(dim), int(nx)
        self.ny = int(ny) if dim == 2 else 1
        self.dx = float(dx)
        self.dy = float(dy if dy is not None else dx) if dim == 2 else float(dx)
        self.precision = precision
        self.device = torch.device(device)
        if precision not in PRECISIONS:
            raise ValueError("precision must be one of %s" % sorted(PRECISIONS))
        # external (host / load_state) element type; "cdf" exchanges complex128
        self.cdtype = torch.complex64 if precision == "c64" else torch.complex128
        self.npdtype = np.complex64 if precision == "c64" else np.complex128
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        self.ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = self.lib.sgpe_init_grid(ctypes.byref(self.ctx), self.dim, self.nx, self.ny, self.dx, self.dy,
                                         PRECISIONS[precision],
                                         ctypes.c_void_p(self.stream.cuda_stream))
        if rc != OK:
            msg = self.lib.sgpe_last_error(None)
            raise SgpeError(rc, "sgpe_init_grid(dim=%d, nx=%d, ny=%d): %s"
                            % (self.dim, self.nx, self.ny, msg.decode() if msg else ""))
        nbytes = ctypes.c_size_t()
        self._check(self.lib.sgpe_workspace_bytes(self.ctx, ctypes.byref(nbytes)))
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        if precision == "cdf":
            # bound state in the double-float pair layout (re_hi, re_lo, im_hi, im_lo)
            self.psi = torch.zeros((3, self.ny, self.nx, 4), dtype=torch.float32, device=self.device)
        else:
            self.psi = torch.zeros((3, self.ny, self.nx), dtype=self.cdtype, device=self.device)
        self._check(self.lib.sgpe_bind(self.ctx, self.psi.data_ptr(), self.workspace.data_ptr()))
        self.physics = None

    def _check(self, rc):
        if rc != OK:
            msg = self.lib.sgpe_last_error(self.ctx)
            raise SgpeError(rc, msg.decode() if msg else "")

    def close(self):
        if self.ctx:
            self.lib.sgpe_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- parameters and state ------------------------------------------------
    def set_params(self, physics: Physics | None = None, **kw):
        if physics is None:
            physics = Physics(**kw)
        self.physics = physics
        p = physics.c()
        self._check(self.lib.sgpe_set_params(self.ctx, ctypes.byref(p)))

    def set_state(self, psi):
        """Upload a host state ([3][ny][nx] complex) through sgpe_set_state."""
        a = np.ascontiguousarray(np.asarray(psi).reshape(3, self.ny, self.nx).astype(self.npdtype))
        self._check(self.lib.sgpe_set_state(self.ctx, a.ctypes.data))

    def set_state_host_ptr(self, ptr: int):
        self._check(self.lib.sgpe_set_state(self.ctx, ctypes.c_void_p(ptr)))

    def load_state(self, psi_dev):
        """Copy a device tensor (same shape and dtype as the state) into the state (sgpe_load_state)."""
        assert psi_dev.is_cuda and psi_dev.dtype == self.cdtype and psi_dev.is_contiguous()
        assert psi_dev.numel() == 3 * self.ny * self.nx
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))
        self._check(self.lib.sgpe_load_state(self.ctx, psi_dev.data_ptr()))

    def get_state(self) -> np.ndarray:
        out = np.empty((3, self.ny, self.nx), dtype=self.npdtype)
        self._check(self.lib.sgpe_get_state(self.ctx, out.ctypes.data))
        return out

    def get_state_host_ptr(self, ptr: int):
        self._check(self.lib.sgpe_get_state(self.ctx, ctypes.c_void_p(ptr)))

    # -- the method ------------------------------------------------------------
    def step_imag(self, nsteps: int):
        self._check(self.lib.sgpe_step_imag(self.ctx, int(nsteps)))

    def step_real(self, nsteps: int, omega_t=None):
        """omega_t: None, or a float64 CUDA tensor with at least nsteps entries."""
        ptr = None
        if omega_t is not None:
            assert omega_t.dtype == self.torch.float64 and omega_t.is_cuda and omega_t.numel() >= nsteps
            self._omega_keep = omega_t
            ptr = omega_t.data_ptr()
        self._check(self.lib.sgpe_step_real(self.ctx, int(nsteps), ptr))

    def substep(self, which: str, imag: bool, omega: float | None = None):
        om = self.physics.omega if omega is None else omega
        self._check(self.lib.sgpe_substep(self.ctx, SUBSTEP[which], int(bool(imag)), float(om)))

    def normalize(self) -> np.ndarray:
        out = np.zeros(3)
        self._check(self.lib.sgpe_normalize(self.ctx, out.ctypes.data))
        return out

    def energy(self) -> dict:
        out = np.zeros(NOBS)
        self._check(self.lib.sgpe_energy(self.ctx, out.ctypes.data))
        return dict(zip(OBS_NAMES, out.tolist()))

    def energy_array(self) -> np.ndarray:
        out = np.zeros(NOBS)
        self._check(self.lib.sgpe_energy(self.ctx, out.ctypes.data))
        return out

    def profile_steps(self, nsteps: int, imag: bool = True):
        """Per-kernel device time (ms, summed) and launch counts over nsteps eager steps."""
        ms = np.zeros(4)
        cnt = np.zeros(4, dtype=np.int32)
        self._check(self.lib.sgpe_profile_steps(self.ctx, int(nsteps), int(bool(imag)), ms.ctypes.data,
                                                cnt.ctypes.data))
        return ms, cnt

    def launches_per_step(self) -> int:
        return int(self.lib.sgpe_launches_per_step(self.ctx))

    def synchronize(self):
        self.stream.synchronize()

    # -- differentiation form ----------------------------------------------------
    def loss_grad(self, omega_t, rho_tgt, checkpoint_every=50):
        """Run len(omega_t) real-time steps from the current state (which ends as
        psi_N) and return (L, dL/dOmega (float64 CUDA tensor), (dL/dwx, dL/dwy))
        for L = cell * sum (rho_N - rho_tgt)^2 (sgpe_adjoint_loss_grad)."""
        torch = self.torch
        om = torch.as_tensor(omega_t, dtype=torch.float64, device=self.device).contiguous()
        tgt = torch.as_tensor(rho_tgt, dtype=torch.float64, device=self.device).reshape(self.ny, self.nx).contiguous()
        n = int(om.numel())
        nb = ctypes.c_size_t()
        self._check(self.lib.sgpe_adjoint_workspace_bytes(self.ctx, n, int(checkpoint_every), ctypes.byref(nb)))
        ws = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)
        dom = torch.zeros(n, dtype=torch.float64, device=self.device)
        L = np.zeros(1)
        dw = np.zeros(2)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        self._check(self.lib.sgpe_adjoint_loss_grad(self.ctx, n, om.data_ptr(), tgt.data_ptr(), int(checkpoint_every),
                                                    ws.data_ptr(), L.ctypes.data, dom.data_ptr(), dw.ctypes.data))
        return float(L[0]), dom, (float(dw[0]), float(dw[1]))

    def adjoint_forward(self, omega_t, checkpoint_every=50):
        """Run len(omega_t) real-time steps from the current state (which ends as
        psi_N), keeping checkpoints for adjoint_step (sgpe_adjoint_forward).
        Returns the tape: the workspace tensor and the Omega table it belongs to."""
        torch = self.torch
        om = torch.as_tensor(omega_t, dtype=torch.float64, device=self.device).contiguous()
        n = int(om.numel())
        nb = ctypes.c_size_t()
        self._check(self.lib.sgpe_adjoint_workspace_bytes(self.ctx, n, int(checkpoint_every), ctypes.byref(nb)))
        ws = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        self._check(self.lib.sgpe_adjoint_forward(self.ctx, n, om.data_ptr(), int(checkpoint_every), ws.data_ptr()))
        return {"ws": ws, "omega": om, "K": int(checkpoint_every)}

    def adjoint_step(self, tape, lam):
        """Reverse the steps of a tape from adjoint_forward for the cotangent
        lam = dL/dpsi_N (device tensor [3][ny][nx] of the state's complex dtype,
        g = dL/dRe + i dL/dIm); returns (dL/dpsi_0, dL/dOmega (float64 tensor),
        (dL/dwx, dL/dwy)) (sgpe_adjoint_step)."""
        torch = self.torch
        om = tape["omega"]
        n = int(om.numel())
        g = lam.detach().to(device=self.device, dtype=self.cdtype).reshape(3, self.ny, self.nx).contiguous().clone()
        dom = torch.zeros(n, dtype=torch.float64, device=self.device)
        dw = np.zeros(2)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        self._check(self.lib.sgpe_adjoint_step(self.ctx, n, om.data_ptr(), tape["K"], tape["ws"].data_ptr(),
                                               g.data_ptr(), dom.data_ptr(), dw.ctypes.data))
        return g, dom, (float(dw[0]), float(dw[1]))


def eval_expm1f(x):
    """exp(x) - 1 of a float32 CUDA tensor by the library's FP32 routine (sgpe_eval_expm1f)."""
    import torch

    lib = load()
    x = x.contiguous()
    if x.dtype != torch.float32 or not x.is_cuda:
        raise ValueError("eval_expm1f takes a float32 CUDA tensor")
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream(x.device)
    rc = lib.sgpe_eval_expm1f(ctypes.c_void_p(stream.cuda_stream), ctypes.c_void_p(x.data_ptr()),
                              ctypes.c_void_p(y.data_ptr()), int(x.numel()))
    if rc != OK:
        msg = lib.sgpe_last_error(None)
        raise SgpeError(rc, msg.decode() if msg else "sgpe_eval_expm1f")
    return y


def measure_fp64_rate(stream=None) -> float:
    """The device's FP64 FMA rate in TFLOP/s (sgpe_measure_fp64_rate)."""
    lib = load()
    out = ctypes.c_double()
    rc = lib.sgpe_measure_fp64_rate(ctypes.c_void_p(stream.cuda_stream if stream is not None else 0),
                                    ctypes.byref(out))
    if rc != OK:
        msg = lib.sgpe_last_error(None)
        raise SgpeError(rc, msg.decode() if msg else "sgpe_measure_fp64_rate")
    return float(out.value)


def _rabi_trap_loss_function():
    import torch

    class RabiTrapLoss(torch.autograd.Function):
        """L(Omega(t), wx, wy) = cell * sum (rho_N - rho_tgt)^2 after real-time
        propagation of psi0 by `solver`; backward uses the library's hand-written
        adjoint (the gradient is computed together with L in forward)."""

        @staticmethod
        def forward(ctx, omega_t, w, solver, psi0, rho_tgt, checkpoint_every=50):
            ph = solver.physics
            solver.set_params(Physics(c0=ph.c0, c2=ph.c2, so_type=ph.so_type, gamma=ph.gamma, omega=ph.omega,
                                      wx=float(w[0]), wy=float(w[1]), dt=ph.dt, renorm=0, mag=ph.mag))
            solver.load_state(psi0)
            L, dom, dw = solver.loss_grad(omega_t.detach(), rho_tgt, checkpoint_every)
            ctx.save_for_backward(dom.to(omega_t.device), torch.tensor(dw, dtype=torch.float64, device=w.device))
            return torch.tensor(L, dtype=torch.float64, device=omega_t.device)

        @staticmethod
        def backward(ctx, grad):
            dom, dw = ctx.saved_tensors
            return grad * dom, grad * dw, None, None, None, None

    return RabiTrapLoss


def _propagate_function():
    import torch

    class RealTimePropagation(torch.autograd.Function):
        """psi_N = S_{N-1} ... S_0 psi_0, the real-time split steps of `solver` with
        Rabi strengths Omega_n and trap frequencies w = (wx, wy): a differentiable
        map of (psi_0, Omega(t), w) whose backward runs the library's adjoint
        (sgpe_adjoint_forward in forward, sgpe_adjoint_step in backward), so any
        loss the caller computes from psi_N can be differentiated."""

        @staticmethod
        def forward(ctx, psi0, omega_t, w, solver, checkpoint_every=50):
            ph = solver.physics
            phys = Physics(c0=ph.c0, c2=ph.c2, so_type=ph.so_type, gamma=ph.gamma, omega=ph.omega,
                           wx=float(w[0]), wy=float(w[1]), dt=ph.dt, renorm=0, mag=ph.mag, split=ph.split,
                           so_mode=ph.so_mode)
            solver.set_params(phys)
            solver.load_state(psi0.detach().contiguous())
            tape = solver.adjoint_forward(omega_t.detach(), checkpoint_every)
            solver.synchronize()
            ctx.solver, ctx.tape, ctx.phys = solver, tape, phys
            ctx.wdev = w.device
            return solver.psi.clone()

        @staticmethod
        def backward(ctx, grad):
            solver = ctx.solver
            if solver.physics != ctx.phys:
                solver.set_params(ctx.phys)
            g0, dom, dw = solver.adjoint_step(ctx.tape, grad)
            solver.synchronize()
            return g0, dom, torch.tensor(dw, dtype=torch.float64, device=ctx.wdev), None, None

    return RealTimePropagation


def propagate_real(psi0, omega_t, w, solver, checkpoint_every=50):
    """Differentiable real-time propagation through the GPU solver (see RealTimePropagation)."""
    return _propagate_function().apply(psi0, omega_t, w, solver, checkpoint_every)


def rabi_trap_loss(omega_t, w, solver, psi0, rho_tgt, checkpoint_every=50):
    """Differentiable loss through the GPU propagator (see RabiTrapLoss)."""
    return _rabi_trap_loss_function().apply(omega_t, w, solver, psi0, rho_tgt, checkpoint_every)


class Instance(ctypes.Structure):
    """sgpe_instance (include/sgpe.h)."""
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("dx", ctypes.c_double),
                ("dy", ctypes.c_double), ("params", Params)]


class BatchSolver:
    """Many independent grids advanced together (sgpe_batch_*); state and workspace are torch tensors."""

    def __init__(self, instances, precision="c128", device="cuda:0", stream=None):
        """instances: list of dicts with dim, nx, ny, dx, dy and the Physics fields."""
        import torch
        self.torch = torch
        self.lib = load()
        self.precision = precision
        self.device = torch.device(device)
        self.cdtype = torch.complex128 if precision == "c128" else torch.complex64
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        self.specs = []
        arr = (Instance * len(instances))()
        for i, d in enumerate(instances):
            dim = int(d["dim"])
            phys = Physics(**{k: d[k] for k in Physics.__dataclass_fields__ if k in d})
            nx, ny = int(d["nx"]), (int(d.get("ny", 1)) if dim == 2 else 1)
            dx = float(d.get("dx", 0.05))
            dy = float(d.get("dy", dx)) if dim == 2 else dx
            arr[i] = Instance(dim, nx, ny, dx, dy, phys.c())
            self.specs.append(dict(dim=dim, nx=nx, ny=ny, dx=dx, dy=dy, physics=phys))
        self.n = len(instances)
        self.b = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = self.lib.sgpe_batch_create(ctypes.byref(self.b), self.n, ctypes.cast(arr, ctypes.c_void_p),
                                            C128 if precision == "c128" else C64,
                                            ctypes.c_void_p(self.stream.cuda_stream))
        if rc != OK:
            msg = self.lib.sgpe_last_error(None)
            raise SgpeError(rc, msg.decode() if msg else "sgpe_batch_create")
        ne, nb = ctypes.c_size_t(), ctypes.c_size_t()
        self._check(self.lib.sgpe_batch_sizes(self.b, ctypes.byref(ne), ctypes.byref(nb)))
        offs = np.zeros(self.n, dtype=np.uint64)
        self._check(self.lib.sgpe_batch_offsets(self.b, offs.ctypes.data))
        self.offsets = [int(o) for o in offs]
        self.psi = torch.zeros(int(ne.value), dtype=self.cdtype, device=self.device)
        self.workspace = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)
        self._check(self.lib.sgpe_batch_bind(self.b, self.psi.data_ptr(), self.workspace.data_ptr()))

    def _check(self, rc):
        if rc != OK:
            msg = self.lib.sgpe_batch_last_error(self.b)
            raise SgpeError(rc, msg.decode() if msg else "")

    def close(self):
        if self.b:
            self.lib.sgpe_batch_destroy(self.b)
            self.b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def view(self, i):
        """Instance i's state as a [3][ny][nx] view of the batch state tensor."""
        s = self.specs[i]
        n = 3 * s["ny"] * s["nx"]
        return self.psi[self.offsets[i]:self.offsets[i] + n].view(3, s["ny"], s["nx"])

    def pack(self, states):
        """Batch state tensor (device) holding the given per-instance host states."""
        out = self.torch.zeros_like(self.psi)
        for i, st in enumerate(states):
            s = self.specs[i]
            n = 3 * s["ny"] * s["nx"]
            out[self.offsets[i]:self.offsets[i] + n] = self.torch.from_numpy(
                np.ascontiguousarray(np.asarray(st).reshape(-1))).to(self.cdtype).to(self.device)
        return out

    def load_state(self, psi_dev):
        assert psi_dev.shape == self.psi.shape and psi_dev.dtype == self.cdtype
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))
        self._check(self.lib.sgpe_batch_load_state(self.b, psi_dev.data_ptr()))

    def step_imag(self, nsteps):
        self._check(self.lib.sgpe_batch_step_imag(self.b, int(nsteps)))

    def step_real(self, nsteps):
        self._check(self.lib.sgpe_batch_step_real(self.b, int(nsteps)))

    def energy(self) -> np.ndarray:
        """(n, NOBS) observables; applies the pending scales to the state."""
        out = np.zeros((self.n, NOBS))
        self._check(self.lib.sgpe_batch_energy(self.b, out.ctypes.data))
        return out

    def states(self):
        """Host copies of every instance's state (call energy() first to apply pending scales)."""
        self.stream.synchronize()
        return [self.view(i).cpu().numpy() for i in range(self.n)]

    def autotune(self, nsteps=4):
        ch = np.zeros(2, dtype=np.int32)
        self._check(self.lib.sgpe_batch_autotune(self.b, int(nsteps), ch.ctypes.data))
        return int(ch[0]), int(ch[1])

    def set_tiles(self, x, y):
        """Launch shape: x part 0 (fused row kernel) or 1/2/4 warps per block of a separate x sweep;
        y sweep 1/2/4 warps per block."""
        self._check(self.lib.sgpe_batch_set_tiles(self.b, int(x), int(y)))

    def launches_per_step(self):
        return int(self.lib.sgpe_batch_launches_per_step(self.b))
