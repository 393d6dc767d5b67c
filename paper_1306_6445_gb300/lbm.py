"""Python binding of the C ABI in include/lb.h (ctypes; argument marshalling only).

Every computation runs in the CUDA library ``_lib/liblb_gb300.so``. When the library
is missing this module raises at first use; there is no CPU fallback.

Low-level functions keep the C names (``lb_init``, ``lb_step``, ``lb_get_rho`` ...).
``Lattice`` wraps one context; by default its two population buffers are device
memory allocated through PyTorch and its work goes to PyTorch's current CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblb_gb300.so")

LB_OK, LB_EINVAL, LB_ENOMEM, LB_ECUDA, LB_ENONFINITE, LB_EDOMAIN, LB_ETIMEOUT = range(7)
STATUS_NAMES = {0: "LB_OK", 1: "LB_EINVAL", 2: "LB_ENOMEM", 3: "LB_ECUDA", 4: "LB_ENONFINITE",
                5: "LB_EDOMAIN", 6: "LB_ETIMEOUT"}
LB_EOS_CS, LB_EOS_EXP, LB_EOS_PIECEWISE = 0, 1, 2
LB_FP64, LB_FP32, LB_BF16 = 0, 1, 2
PRECS = {"fp64": LB_FP64, "fp32": LB_FP32, "bf16": LB_BF16}
LB_BC_PERIODIC, LB_BC_WALLS_Y, LB_BC_OPEN = 0, 1, 2

# every exported symbol of include/lb.h
EXPORTED = ["lb_pitch", "lb_buffer_bytes", "lb_init", "lb_init_ex", "lb_set_rho_u", "lb_step",
            "lb_sync", "lb_get_rho", "lb_get_u", "lb_get_populations", "lb_set_populations",
            "lb_reduce", "lb_steps_done", "lb_kernels_per_step", "lb_last_error",
            "lb_status_of", "lb_free", "lb_cs_critical", "lb_maxwell", "lb_launch_variants",
            "lb_probe_fp64_fma_rate", "lb_measure_droplet", "lb_interface_height",
            "lb_set_launch", "lb_get_launch", "lb_debug_stall_row", "lb_reduce_noalloc",
            "lb_autotune", "lb_set_storage_shift", "lb_set_viscosity_switch",
            "lb_set_storage_rounding",
            "lb_batch_create", "lb_batch_set_rho_u", "lb_batch_step", "lb_batch_sync",
            "lb_batch_errors", "lb_batch_get_rho", "lb_batch_get_populations", "lb_batch_measure",
            "lb_batch_autotune", "lb_batch_set_launch", "lb_batch_get_launch",
            "lb_batch_steps_done", "lb_batch_size", "lb_batch_last_error", "lb_batch_free",
            "lb_batch_set_active", "lb_batch_lattice_steps",
            "lb_strip_widths",
            # include/lb_mlp.h
            "lb_mlp_create", "lb_mlp_set_params", "lb_mlp_get_params", "lb_mlp_set_data",
            "lb_mlp_get_norm", "lb_mlp_set_norm", "lb_mlp_loss_grad", "lb_mlp_train",
            "lb_mlp_steps_done", "lb_mlp_forward", "lb_mlp_invert_kappa", "lb_mlp_last_error",
            "lb_mlp_free"]
MLP_PARAMS = 4611


class LBError(RuntimeError):
    def __init__(self, status: int, where: str, message: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} {message}".rstrip())


class c_lb_eos(C.Structure):
    _fields_ = [("kind", C.c_int), ("a", C.c_double), ("b", C.c_double), ("R", C.c_double),
                ("T", C.c_double), ("psi0", C.c_double), ("rho0", C.c_double),
                ("theta_v", C.c_double), ("theta_m", C.c_double), ("theta_l", C.c_double),
                ("rho1", C.c_double), ("rho2", C.c_double)]


class c_lb_rates(C.Structure):
    _fields_ = [("s_rho", C.c_double), ("s_e", C.c_double), ("s_zeta", C.c_double),
                ("s_j", C.c_double), ("s_q", C.c_double), ("s_v", C.c_double)]


class c_lb_lattice_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("eos", c_lb_eos), ("G", C.c_double),
                ("kappa", C.c_double), ("sigma_force", C.c_double), ("rates", c_lb_rates)]


class c_lb_mlp_norm(C.Structure):
    _fields_ = [("in_mean", C.c_float * 3), ("in_scale", C.c_float * 3),
                ("out_mean", C.c_float * 3), ("out_scale", C.c_float * 3)]


_lib = None


def load_library():
    """Load the CUDA library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library missing ({LIB_PATH}); build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(LIB_PATH)
    P, I, D, SZ = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    DP = C.POINTER(C.c_double)
    F, FP = C.c_float, C.POINTER(C.c_float)
    sig = {
        "lb_pitch": (SZ, [I, I]),
        "lb_buffer_bytes": (SZ, [I, I, I]),
        "lb_init": (I, [C.POINTER(P), I, I, C.POINTER(c_lb_eos), D, D, D, C.POINTER(c_lb_rates),
                        I, I, P]),
        "lb_init_ex": (I, [C.POINTER(P), I, I, C.POINTER(c_lb_eos), D, D, D,
                           C.POINTER(c_lb_rates), I, I, P, P, P]),
        "lb_set_rho_u": (I, [P, DP, DP, DP]),
        "lb_step": (I, [P, I]),
        "lb_sync": (I, [P]),
        "lb_get_rho": (I, [P, DP]),
        "lb_get_u": (I, [P, DP, DP]),
        "lb_get_populations": (I, [P, P, SZ]),
        "lb_set_populations": (I, [P, P, SZ]),
        "lb_reduce": (I, [P, DP]),
        "lb_steps_done": (C.c_longlong, [P]),
        "lb_kernels_per_step": (I, [P]),
        "lb_last_error": (C.c_char_p, [P]),
        "lb_status_of": (I, [P]),
        "lb_free": (None, [P]),
        "lb_cs_critical": (I, [D, D, D, DP, DP]),
        "lb_maxwell": (I, [C.POINTER(c_lb_eos), D, DP, DP, DP]),
        "lb_probe_fp64_fma_rate": (I, [P, I, DP]),
        "lb_measure_droplet": (I, [P, D, DP]),
        "lb_interface_height": (I, [P, D, DP]),
        "lb_launch_variants": (I, []),
        "lb_set_launch": (I, [P, I, I]),
        "lb_autotune": (I, [P, I, C.POINTER(I), C.POINTER(I)]),
        "lb_set_storage_shift": (I, [P, D]),
        "lb_set_storage_rounding": (I, [P, I]),
        "lb_set_viscosity_switch": (I, [P, D, D]),
        "lb_get_launch": (I, [P, C.POINTER(I), C.POINTER(I), C.POINTER(I), C.POINTER(I)]),
        "lb_debug_stall_row": (I, [P, I]),
        "lb_reduce_noalloc": (I, [P, DP]),
        "lb_batch_create": (I, [C.POINTER(P), I, C.POINTER(c_lb_lattice_desc), I, P]),
        "lb_batch_set_rho_u": (I, [P, I, DP, DP, DP]),
        "lb_batch_step": (I, [P, I]),
        "lb_batch_sync": (I, [P]),
        "lb_batch_errors": (I, [P, C.POINTER(I)]),
        "lb_batch_get_rho": (I, [P, I, DP]),
        "lb_batch_get_populations": (I, [P, I, P, SZ]),
        "lb_batch_measure": (I, [P, DP, DP]),
        "lb_batch_autotune": (I, [P, I, C.POINTER(I), C.POINTER(I)]),
        "lb_batch_set_launch": (I, [P, I, I]),
        "lb_batch_get_launch": (I, [P, C.POINTER(I), C.POINTER(I), C.POINTER(I), C.POINTER(I)]),
        "lb_batch_steps_done": (C.c_longlong, [P]),
        "lb_batch_set_active": (I, [P, C.POINTER(C.c_ubyte)]),
        "lb_batch_lattice_steps": (C.c_longlong, [P, I]),
        "lb_batch_size": (I, [P]),
        "lb_batch_last_error": (C.c_char_p, [P]),
        "lb_batch_free": (None, [P]),
        "lb_strip_widths": (I, [I, I, C.POINTER(I), I]),
        "lb_mlp_create": (I, [C.POINTER(P), I, P]),
        "lb_mlp_set_params": (I, [P, FP]),
        "lb_mlp_get_params": (I, [P, FP]),
        "lb_mlp_set_data": (I, [P, FP, FP, I]),
        "lb_mlp_get_norm": (I, [P, C.POINTER(c_lb_mlp_norm)]),
        "lb_mlp_set_norm": (I, [P, C.POINTER(c_lb_mlp_norm)]),
        "lb_mlp_loss_grad": (I, [P, FP, FP]),
        "lb_mlp_train": (I, [P, I, F, F, F, F, FP]),
        "lb_mlp_steps_done": (C.c_longlong, [P]),
        "lb_mlp_forward": (I, [P, FP, FP, I]),
        "lb_mlp_invert_kappa": (I, [P, FP, I, F, F, FP]),
        "lb_mlp_last_error": (C.c_char_p, [P]),
        "lb_mlp_free": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _check(status: int, where: str, ctx=None):
    if status != LB_OK:
        msg = ""
        if ctx is not None:
            raw = load_library().lb_last_error(ctx)
            msg = raw.decode() if raw else ""
        raise LBError(status, where, msg)


# ------------------------------------------------------------------------------------
# parameters
# ------------------------------------------------------------------------------------

@dataclass(frozen=True)
class EOSParams:
    """Mirror of lb_eos. kind: "cs" | "exp" | "piecewise"."""

    kind: str = "cs"
    a: float = 1.0
    b: float = 4.0
    R: float = 1.0
    T: float = 0.0
    psi0: float = 4.0
    rho0: float = 200.0
    theta_v: float = 0.49 / 3.0
    theta_m: float = -0.06 / 3.0
    theta_l: float = 1.0 / 3.0
    rho1: float = 1.49
    rho2: float = 94.65

    def to_c(self) -> c_lb_eos:
        kinds = {"cs": LB_EOS_CS, "exp": LB_EOS_EXP, "piecewise": LB_EOS_PIECEWISE}
        return c_lb_eos(kinds[self.kind], self.a, self.b, self.R, self.T, self.psi0, self.rho0,
                        self.theta_v, self.theta_m, self.theta_l, self.rho1, self.rho2)


@dataclass(frozen=True)
class RateParams:
    """Mirror of lb_rates (s = 1/tau)."""

    s_rho: float = 1.0
    s_e: float = 0.8
    s_zeta: float = 0.8
    s_j: float = 1.0
    s_q: float = 1.1
    s_v: float = 1.0 / 0.8

    def to_c(self) -> c_lb_rates:
        return c_lb_rates(self.s_rho, self.s_e, self.s_zeta, self.s_j, self.s_q, self.s_v)

    @staticmethod
    def from_viscosity(nu: float, **kw) -> "RateParams":
        return RateParams(s_v=1.0 / (3.0 * nu + 0.5), **kw)


def lb_cs_critical(a: float = 1.0, b: float = 4.0, R: float = 1.0):
    Tc, rc = C.c_double(), C.c_double()
    _check(load_library().lb_cs_critical(a, b, R, C.byref(Tc), C.byref(rc)), "lb_cs_critical")
    return Tc.value, rc.value


def cs_eos(t_over_tc: float, a: float = 1.0, b: float = 4.0, R: float = 1.0) -> EOSParams:
    Tc, _ = lb_cs_critical(a, b, R)
    return EOSParams(kind="cs", a=a, b=b, R=R, T=t_over_tc * Tc)


def lb_maxwell(eos: EOSParams, G: float):
    rv, rl, pb = C.c_double(), C.c_double(), C.c_double()
    e = eos.to_c()
    _check(load_library().lb_maxwell(C.byref(e), G, C.byref(rv), C.byref(rl), C.byref(pb)),
           "lb_maxwell")
    return rv.value, rl.value, pb.value


def lb_probe_fp64_fma_rate(stream=None, iters: int = 4096) -> float:
    """FP64 FMA thread instructions per second of the current device (the ALU roof of the
    FP64 update); `stream` a cudaStream_t handle (int) or None for the default stream."""
    r = C.c_double()
    _check(load_library().lb_probe_fp64_fma_rate(C.c_void_p(stream or 0), iters, C.byref(r)),
           "lb_probe_fp64_fma_rate")
    return r.value


def lb_pitch(nx: int, prec: int) -> int:
    return int(load_library().lb_pitch(nx, prec))


def lb_buffer_bytes(nx: int, ny: int, prec: int) -> int:
    return int(load_library().lb_buffer_bytes(nx, ny, prec))


# ------------------------------------------------------------------------------------
# context wrappers with the C names
# ------------------------------------------------------------------------------------

def lb_init(nx, ny, eos: EOSParams, G, kappa, sigma_force, rates: RateParams, prec, bc,
            stream=None):
    lib = load_library()
    ctx = C.c_void_p()
    e, r = eos.to_c(), rates.to_c()
    _check(lib.lb_init(C.byref(ctx), nx, ny, C.byref(e), G, kappa, sigma_force, C.byref(r),
                       prec, bc, stream), "lb_init")
    return ctx


def lb_init_ex(nx, ny, eos: EOSParams, G, kappa, sigma_force, rates: RateParams, prec, bc,
               stream, f_a_ptr: int, f_b_ptr: int):
    lib = load_library()
    ctx = C.c_void_p()
    e, r = eos.to_c(), rates.to_c()
    _check(lib.lb_init_ex(C.byref(ctx), nx, ny, C.byref(e), G, kappa, sigma_force, C.byref(r),
                          prec, bc, stream, C.c_void_p(f_a_ptr), C.c_void_p(f_b_ptr)),
           "lb_init_ex")
    return ctx


def lb_set_rho_u(ctx, rho, ux, uy):
    rho, ux, uy = (np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy))
    _check(load_library().lb_set_rho_u(ctx, _dp(rho), _dp(ux), _dp(uy)), "lb_set_rho_u", ctx)


def lb_step(ctx, n: int):
    _check(load_library().lb_step(ctx, int(n)), "lb_step", ctx)


def lb_sync(ctx):
    _check(load_library().lb_sync(ctx), "lb_sync", ctx)


def lb_get_rho(ctx, out: np.ndarray):
    _check(load_library().lb_get_rho(ctx, _dp(out)), "lb_get_rho", ctx)
    return out


def lb_get_u(ctx, ux: np.ndarray, uy: np.ndarray):
    _check(load_library().lb_get_u(ctx, _dp(ux), _dp(uy)), "lb_get_u", ctx)
    return ux, uy


def lb_get_populations(ctx, dst_ptr: int, nbytes: int):
    _check(load_library().lb_get_populations(ctx, C.c_void_p(dst_ptr), nbytes),
           "lb_get_populations", ctx)


def lb_set_populations(ctx, src_ptr: int, nbytes: int):
    _check(load_library().lb_set_populations(ctx, C.c_void_p(src_ptr), nbytes),
           "lb_set_populations", ctx)


def lb_reduce(ctx):
    out = np.zeros(4)
    _check(load_library().lb_reduce(ctx, _dp(out)), "lb_reduce", ctx)
    return out


def lb_measure_droplet(ctx, radius: float):
    """Laplace-law measurement on the GPU (see include/lb.h): a dict with theta, rho_in,
    rho_out, R, p_in, p_out, mass, failed."""
    out = np.zeros(8)
    _check(load_library().lb_measure_droplet(ctx, float(radius), _dp(out)), "lb_measure_droplet",
           ctx)
    keys = ("theta", "rho_in", "rho_out", "R", "p_in", "p_out", "mass", "failed")
    return dict(zip(keys, out.tolist()))


def lb_interface_height(ctx, rho_mid: float, nx: int):
    """Interface height of every column (nx doubles, NaN where there is none)."""
    out = np.zeros(nx)
    _check(load_library().lb_interface_height(ctx, float(rho_mid), _dp(out)),
           "lb_interface_height", ctx)
    return out


def lb_reduce_noalloc(ctx):
    """lb_reduce without device allocation (static scratch); see include/lb.h."""
    out = np.zeros(4)
    _check(load_library().lb_reduce_noalloc(ctx, _dp(out)), "lb_reduce_noalloc", ctx)
    return out


def lb_steps_done(ctx) -> int:
    return int(load_library().lb_steps_done(ctx))


def lb_kernels_per_step(ctx) -> int:
    return int(load_library().lb_kernels_per_step(ctx))


def lb_launch_variants() -> int:
    return int(load_library().lb_launch_variants())


def lb_set_launch(ctx, variant: int, rows: int = 0):
    _check(load_library().lb_set_launch(ctx, int(variant), int(rows)), "lb_set_launch", ctx)


def lb_autotune(ctx, trial_steps: int = 5):
    v, r = C.c_int(), C.c_int()
    _check(load_library().lb_autotune(ctx, trial_steps, C.byref(v), C.byref(r)), "lb_autotune",
           ctx)
    return v.value, r.value


def lb_set_viscosity_switch(ctx, rho_1: float, s_v_vapour: float):
    _check(load_library().lb_set_viscosity_switch(ctx, float(rho_1), float(s_v_vapour)),
           "lb_set_viscosity_switch", ctx)


LB_ROUND_NEAREST, LB_ROUND_STOCHASTIC = 0, 1


def lb_set_storage_rounding(ctx, mode: int):
    _check(load_library().lb_set_storage_rounding(ctx, int(mode)), "lb_set_storage_rounding", ctx)


def lb_set_storage_shift(ctx, rho_s: float):
    _check(load_library().lb_set_storage_shift(ctx, float(rho_s)), "lb_set_storage_shift", ctx)


def lb_get_launch(ctx):
    v, tx, rows, occ = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    _check(load_library().lb_get_launch(ctx, C.byref(v), C.byref(tx), C.byref(rows),
                                        C.byref(occ)), "lb_get_launch")
    return {"variant": v.value, "tx": tx.value, "rows": rows.value, "ctas_per_sm": occ.value}


def lb_debug_stall_row(ctx, row: int):
    _check(load_library().lb_debug_stall_row(ctx, int(row)), "lb_debug_stall_row", ctx)


def lb_status_of(ctx) -> int:
    return int(load_library().lb_status_of(ctx))


def lb_last_error(ctx) -> str:
    raw = load_library().lb_last_error(ctx)
    return raw.decode() if raw else ""


def lb_free(ctx):
    if ctx:
        load_library().lb_free(ctx)


# ------------------------------------------------------------------------------------
# convenience wrapper
# ------------------------------------------------------------------------------------

@dataclass
class Lattice:
    """One lattice on the current CUDA device.

    buffers="torch": the two population buffers are torch uint8 device tensors and the
    work runs on torch's current stream (lb_init_ex). buffers="library": lb_init
    allocates them and uses the legacy default stream."""

    nx: int
    ny: int
    eos: EOSParams
    G: float
    kappa: float = 0.0
    sigma_force: float = 0.0
    rates: RateParams = field(default_factory=RateParams)
    prec: str = "fp64"
    walls_y: bool = False
    buffers: str = "torch"
    storage_shift: float = 0.0   # rho_s of prec="bf16" (stored BF16 of f_a - w_a rho_s)
    stochastic_rounding: bool = False   # prec="bf16": LB_ROUND_STOCHASTIC
    open_bc: bool = False         # LB_BC_OPEN: wall below, open top and sides (Sec. V.C)
    viscosity_switch: tuple = None   # (rho_1, s_v where rho < rho_1), LB_BC_OPEN only

    def __post_init__(self):
        if self.prec not in PRECS:
            raise LBError(LB_EINVAL, "Lattice", f"prec must be one of {sorted(PRECS)}")
        self._prec = PRECS[self.prec]
        # host population arrays: float64 / float32, or the raw 16-bit patterns for bf16
        self.dtype = {LB_FP64: np.float64, LB_FP32: np.float32, LB_BF16: np.uint16}[self._prec]
        if self.walls_y and self.open_bc:
            raise LBError(LB_EINVAL, "Lattice", "walls_y and open_bc exclude each other")
        bc = LB_BC_OPEN if self.open_bc else (LB_BC_WALLS_Y if self.walls_y else LB_BC_PERIODIC)
        self._tensors = None
        if self.buffers == "torch":
            import torch
            nbytes = lb_buffer_bytes(self.nx, self.ny, self._prec)
            a = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            b = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            self._tensors = (a, b)
            self.stream = torch.cuda.current_stream().cuda_stream
            self.ctx = lb_init_ex(self.nx, self.ny, self.eos, self.G, self.kappa,
                                  self.sigma_force, self.rates, self._prec, bc, self.stream,
                                  a.data_ptr(), b.data_ptr())
        else:
            self.stream = None
            self.ctx = lb_init(self.nx, self.ny, self.eos, self.G, self.kappa, self.sigma_force,
                               self.rates, self._prec, bc, None)
        if self._prec == LB_BF16:
            lb_set_storage_shift(self.ctx, self.storage_shift)
            if self.stochastic_rounding:
                lb_set_storage_rounding(self.ctx, LB_ROUND_STOCHASTIC)
        if self.viscosity_switch is not None:
            lb_set_viscosity_switch(self.ctx, *self.viscosity_switch)

    # --- state
    def set_rho_u(self, rho, ux=None, uy=None):
        z = np.zeros((self.ny, self.nx))
        lb_set_rho_u(self.ctx, rho, z if ux is None else ux, z if uy is None else uy)

    def set_populations(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=self.dtype)
        assert f.shape == (9, self.ny, self.nx)
        lb_set_populations(self.ctx, f.ctypes.data, f.nbytes)

    def populations(self) -> np.ndarray:
        out = np.empty((9, self.ny, self.nx), dtype=self.dtype)
        lb_get_populations(self.ctx, out.ctypes.data, out.nbytes)
        return out

    # --- time stepping and diagnostics
    def autotune(self, trial_steps: int = 5):
        """Pick the fastest step-kernel launch for this lattice (state unchanged)."""
        return lb_autotune(self.ctx, trial_steps)

    def step(self, n: int = 1):
        lb_step(self.ctx, n)

    def sync(self):
        lb_sync(self.ctx)

    def rho(self) -> np.ndarray:
        return lb_get_rho(self.ctx, np.empty((self.ny, self.nx)))

    def u(self):
        return lb_get_u(self.ctx, np.empty((self.ny, self.nx)), np.empty((self.ny, self.nx)))

    def reduce(self) -> np.ndarray:
        return lb_reduce(self.ctx)

    def measure_droplet(self, radius: float) -> dict:
        return lb_measure_droplet(self.ctx, radius)

    def interface_height(self, rho_mid: float) -> np.ndarray:
        return lb_interface_height(self.ctx, rho_mid, self.nx)

    @property
    def steps_done(self) -> int:
        return lb_steps_done(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            lb_free(self.ctx)
            self.ctx = None
        self._tensors = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------------------------
# batched lattices
# ------------------------------------------------------------------------------------

@dataclass(frozen=True)
class LatticeDesc:
    """One lattice of a batch (periodic): size and parameters as in lb_init."""

    nx: int
    ny: int
    eos: EOSParams
    G: float
    kappa: float = 0.0
    sigma_force: float = 0.0
    rates: RateParams = field(default_factory=RateParams)

    def to_c(self) -> c_lb_lattice_desc:
        return c_lb_lattice_desc(self.nx, self.ny, self.eos.to_c(), self.G, self.kappa,
                                 self.sigma_force, self.rates.to_c())


def _bcheck(status: int, where: str, b=None):
    if status != LB_OK:
        msg = ""
        if b is not None:
            raw = load_library().lb_batch_last_error(b)
            msg = raw.decode() if raw else ""
        raise LBError(status, where, msg)


def lb_strip_widths(nx: int, tx: int):
    out = (C.c_int * 4096)()
    n = load_library().lb_strip_widths(nx, tx, out, 4096)
    if n < 0:
        raise LBError(LB_EINVAL, "lb_strip_widths")
    return list(out[:n])


class Batch:
    """Many periodic lattices advanced together (lb_batch_*), on torch's current stream."""

    def __init__(self, descs, prec: str = "fp32", stream=None):
        lib = load_library()
        self.descs = list(descs)
        self.n = len(self.descs)
        if prec not in ("fp32", "fp64"):
            raise LBError(LB_EINVAL, "Batch", "batches are fp32 or fp64")
        self._prec = LB_FP32 if prec == "fp32" else LB_FP64
        self.dtype = np.float32 if self._prec == LB_FP32 else np.float64
        arr = (c_lb_lattice_desc * self.n)(*[d.to_c() for d in self.descs])
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.b = C.c_void_p()
        _bcheck(lib.lb_batch_create(C.byref(self.b), self.n, arr, self._prec, stream),
                "lb_batch_create")

    def set_rho_u(self, i, rho, ux=None, uy=None):
        d = self.descs[i]
        z = np.zeros((d.ny, d.nx))
        rho, ux, uy = (np.ascontiguousarray(a, dtype=np.float64)
                       for a in (rho, z if ux is None else ux, z if uy is None else uy))
        _bcheck(load_library().lb_batch_set_rho_u(self.b, i, _dp(rho), _dp(ux), _dp(uy)),
                "lb_batch_set_rho_u", self.b)

    def step(self, n: int):
        _bcheck(load_library().lb_batch_step(self.b, int(n)), "lb_batch_step", self.b)

    def sync(self):
        _bcheck(load_library().lb_batch_sync(self.b), "lb_batch_sync", self.b)

    def errors(self) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.int32)
        st = load_library().lb_batch_errors(self.b, out.ctypes.data_as(C.POINTER(C.c_int)))
        if st not in (LB_OK, LB_ETIMEOUT):
            _bcheck(st, "lb_batch_errors", self.b)
        return out

    def rho(self, i) -> np.ndarray:
        d = self.descs[i]
        out = np.empty((d.ny, d.nx))
        _bcheck(load_library().lb_batch_get_rho(self.b, i, _dp(out)), "lb_batch_get_rho", self.b)
        return out

    def populations(self, i) -> np.ndarray:
        d = self.descs[i]
        out = np.empty((9, d.ny, d.nx), dtype=self.dtype)
        _bcheck(load_library().lb_batch_get_populations(self.b, i, C.c_void_p(out.ctypes.data),
                                                        out.nbytes),
                "lb_batch_get_populations", self.b)
        return out

    def measure(self, radius) -> np.ndarray:
        """Per lattice: theta, rho_in, rho_out, R, p_in, p_out, mass, failed (n x 8)."""
        r = np.ascontiguousarray(radius, dtype=np.float64)
        out = np.zeros((self.n, 8))
        _bcheck(load_library().lb_batch_measure(self.b, _dp(r), _dp(out)), "lb_batch_measure",
                self.b)
        return out

    def autotune(self, trial_steps: int = 4):
        v, r = C.c_int(), C.c_int()
        _bcheck(load_library().lb_batch_autotune(self.b, trial_steps, C.byref(v), C.byref(r)),
                "lb_batch_autotune", self.b)
        return v.value, r.value

    def set_launch(self, variant: int, rows: int):
        _bcheck(load_library().lb_batch_set_launch(self.b, variant, rows), "lb_batch_set_launch",
                self.b)

    def launch(self):
        v, r, g, n = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        _bcheck(load_library().lb_batch_get_launch(self.b, C.byref(v), C.byref(r), C.byref(g),
                                                   C.byref(n)), "lb_batch_get_launch")
        return {"variant": v.value, "rows": r.value, "grid": g.value, "items": n.value}

    @property
    def steps_done(self) -> int:
        return int(load_library().lb_batch_steps_done(self.b))

    def set_active(self, active):
        """Which lattices lb_batch_step advances (a boolean per lattice); see include/lb.h."""
        a = np.ascontiguousarray(np.asarray(active, dtype=bool), dtype=np.uint8)
        if a.shape != (self.n,):
            raise LBError(LB_EINVAL, "set_active", f"need {self.n} flags")
        _bcheck(load_library().lb_batch_set_active(self.b, a.ctypes.data_as(C.POINTER(C.c_ubyte))),
                "lb_batch_set_active", self.b)

    def lattice_steps(self, i: int) -> int:
        return int(load_library().lb_batch_lattice_steps(self.b, int(i)))

    def close(self):
        if getattr(self, "b", None):
            load_library().lb_batch_free(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------------------------
# surrogate network (include/lb_mlp.h)
# ------------------------------------------------------------------------------------

def _fp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _f32(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a if shape is None else a.reshape(shape)


class MLP:
    """The 3-64-64-3 surrogate (T/T_c, kappa, tau_v) -> (sigma, rho_l, rho_v), trained and
    evaluated by the library's kernels (lb_mlp_*), on torch's current stream."""

    def __init__(self, max_samples: int = 4096, stream=None):
        lib = load_library()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.m = C.c_void_p()
        self._check(lib.lb_mlp_create(C.byref(self.m), int(max_samples), stream),
                    "lb_mlp_create")

    def _check(self, status, where):
        if status != LB_OK:
            msg = ""
            if getattr(self, "m", None):
                raw = load_library().lb_mlp_last_error(self.m)
                msg = raw.decode() if raw else ""
            raise LBError(status, where, msg)

    def set_params(self, params):
        p = _f32(params)
        if p.size != MLP_PARAMS:
            raise LBError(LB_EINVAL, "lb_mlp_set_params", f"need {MLP_PARAMS} values")
        self._check(load_library().lb_mlp_set_params(self.m, _fp(p)), "lb_mlp_set_params")

    def params(self) -> np.ndarray:
        out = np.empty(MLP_PARAMS, dtype=np.float32)
        self._check(load_library().lb_mlp_get_params(self.m, _fp(out)), "lb_mlp_get_params")
        return out

    def set_data(self, x, y):
        x, y = _f32(x), _f32(y)
        if x.ndim != 2 or x.shape[1] != 3 or y.shape != x.shape:
            raise LBError(LB_EINVAL, "lb_mlp_set_data", "x and y must be n x 3")
        self._check(load_library().lb_mlp_set_data(self.m, _fp(x), _fp(y), x.shape[0]),
                    "lb_mlp_set_data")

    def norm(self):
        nm = c_lb_mlp_norm()
        self._check(load_library().lb_mlp_get_norm(self.m, C.byref(nm)), "lb_mlp_get_norm")
        return tuple(np.array(list(getattr(nm, f)), dtype=np.float32)
                     for f in ("in_mean", "in_scale", "out_mean", "out_scale"))

    def set_norm(self, norm):
        nm = c_lb_mlp_norm()
        for f, v in zip(("in_mean", "in_scale", "out_mean", "out_scale"), norm):
            getattr(nm, f)[:] = [float(t) for t in v]
        self._check(load_library().lb_mlp_set_norm(self.m, C.byref(nm)), "lb_mlp_set_norm")

    def loss_grad(self):
        loss = C.c_float()
        g = np.empty(MLP_PARAMS, dtype=np.float32)
        self._check(load_library().lb_mlp_loss_grad(self.m, C.byref(loss), _fp(g)),
                    "lb_mlp_loss_grad")
        return loss.value, g

    def train(self, steps: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8) -> float:
        loss = C.c_float()
        self._check(load_library().lb_mlp_train(self.m, int(steps), lr, beta1, beta2, eps,
                                                C.byref(loss)), "lb_mlp_train")
        return loss.value

    @property
    def steps_done(self) -> int:
        return int(load_library().lb_mlp_steps_done(self.m))

    def forward(self, x) -> np.ndarray:
        x = _f32(x)
        n = x.shape[0]
        y = np.empty((n, 3), dtype=np.float32)
        self._check(load_library().lb_mlp_forward(self.m, _fp(x), _fp(y), n), "lb_mlp_forward")
        return y

    def invert_kappa(self, queries, kappa_lo: float = 0.0, kappa_hi: float = 0.95) -> np.ndarray:
        """queries: n x 3 of (T/T_c, tau_v, sigma_target); NaN where not bracketed."""
        q = _f32(queries)
        n = q.shape[0]
        out = np.empty(n, dtype=np.float32)
        self._check(load_library().lb_mlp_invert_kappa(self.m, _fp(q), n, kappa_lo, kappa_hi,
                                                       _fp(out)), "lb_mlp_invert_kappa")
        return out

    def close(self):
        if getattr(self, "m", None):
            load_library().lb_mlp_free(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
