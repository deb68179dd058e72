"""ctypes binding of include/firm.h: same names, argument marshalling only.

Arrays may be torch tensors (CPU or CUDA) or numpy arrays; the library decides
from the pointer whether memory is host or device.  Every step of the
computation runs inside libfirm.so; nothing here computes.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfirm.so")

(FIRM_OK, FIRM_EINVAL, FIRM_ENOMEM, FIRM_ECUDA, FIRM_ENOTCONV, FIRM_EBREAKDOWN, FIRM_ETIMEOUT, FIRM_ESTATE,
 FIRM_EINTERNAL) = range(9)
FIRM_IMG_F32, FIRM_IMG_BF16 = 0, 1
FIRM_LAMBDA_RELATIVE, FIRM_LAMBDA_ABSOLUTE = 0, 1
FIRM_OUT_KER, FIRM_OUT_KHAT, FIRM_OUT_RHS, FIRM_OUT_SAMPLES, FIRM_OUT_BIN_IDS, FIRM_OUT_BIN_WORK = 0, 1, 2, 3, 4, 5
FIRM_PRECOND_NONE, FIRM_PRECOND_CIRCULANT, FIRM_PRECOND_BINNED, FIRM_PRECOND_TABLE = 0, 1, 2, 3
FIRM_BATCH_GRAPH, FIRM_BATCH_PERSISTENT, FIRM_BATCH_LEARNED = 1, 2, 4
FIRM_FLAG_FP64_CG, FIRM_FLAG_FUSED = 1, 2

EXPORTED = [
    "firm_workspace_size", "firm_plan", "firm_kernel", "firm_backproject", "firm_kernel_backproject", "firm_load_sums",
    "firm_stage_images", "firm_cg_solve",
    "firm_forward", "firm_data_residual", "firm_set_damping", "firm_solve_nonneg",
    "firm_toeplitz_apply", "firm_toeplitz_apply_static", "firm_set_precond", "firm_lambda_eff", "firm_copy_out", "firm_set_timing",
    "firm_stage_times", "firm_launch_count", "firm_pc_features", "firm_pc_net_input", "firm_pc_target", "firm_pc_axis",
    "firm_set_precond_table", "firm_pc_bin_volumes", "firm_pc_baseline", "firm_pc_residual_target", "firm_set_precond_residual",
    "firm_mlp_forward", "firm_mlp_to_bf16", "firm_mlp_forward_bf16", "firm_mlp_grad",
    "firm_mlp_adam", "firm_mlp_param_count", "firm_mlp_work_floats",
    "firm_bin", "firm_bin_info",
    "firm_batch_workspace_size", "firm_batch_create", "firm_batch_run", "firm_batch_solve", "firm_batch_set_network",
    "firm_batch_wait", "firm_batch_set_config",
    "firm_batch_get_config", "firm_batch_tune", "firm_batch_launch_count", "firm_batch_destroy",
    "firm_destroy", "firm_strerror",
]


class firm_ctf_group(ctypes.Structure):
    _fields_ = [("defocus_A", ctypes.c_double), ("kV", ctypes.c_double), ("Cs_mm", ctypes.c_double),
                ("amp_contrast", ctypes.c_double), ("pixel_A", ctypes.c_double),
                ("bfactor_A2", ctypes.c_double)]


class firm_params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("M", ctypes.c_int), ("n_groups", ctypes.c_int), ("W", ctypes.c_int),
                ("sigma", ctypes.c_double), ("lambda_", ctypes.c_double), ("lambda_mode", ctypes.c_int),
                ("disc_mode", ctypes.c_int), ("img_dtype", ctypes.c_int), ("flags", ctypes.c_int)]


class firm_batch_item(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("R", ctypes.c_void_p), ("group", ctypes.c_void_p), ("images", ctypes.c_void_p),
                ("shifts", ctypes.c_void_p), ("x", ctypes.c_void_p)]


class FirmError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} (status {code})")
        self.code = code


_lib = None


def lib() -> ctypes.CDLL:
    """Load libfirm.so (built by __graft_entry__.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.firm_workspace_size.argtypes = [ctypes.POINTER(firm_params), ctypes.POINTER(ctypes.c_size_t)]
    L.firm_plan.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(firm_params), ctypes.POINTER(firm_ctf_group),
                            vp, ctypes.c_size_t, vp]
    L.firm_kernel.argtypes = [vp, i, vp, vp, vp]
    L.firm_backproject.argtypes = [vp, i, vp, vp, vp, vp, vp]
    L.firm_kernel_backproject.argtypes = [vp, i, vp, vp, vp, vp, vp, vp]
    L.firm_load_sums.argtypes = [vp, vp, vp]
    L.firm_stage_images.argtypes = [vp, i, vp, vp, ctypes.c_size_t]
    L.firm_forward.argtypes = [vp, i, vp, vp, vp, vp]
    L.firm_set_damping.argtypes = [vp, d]
    L.firm_solve_nonneg.argtypes = [vp, vp, i, d, ctypes.POINTER(i)]
    L.firm_data_residual.argtypes = [vp, i, vp, vp, vp, vp, vp, vp]
    L.firm_cg_solve.argtypes = [vp, vp, vp, i, d, vp, ctypes.POINTER(i)]
    L.firm_toeplitz_apply.argtypes = [vp, vp, vp]
    L.firm_toeplitz_apply_static.argtypes = [i, vp, d, vp, vp, vp]
    L.firm_set_precond.argtypes = [vp, i]
    L.firm_lambda_eff.argtypes = [vp, ctypes.POINTER(d)]
    L.firm_copy_out.argtypes = [vp, i, vp]
    L.firm_set_timing.argtypes = [vp, i]
    L.firm_stage_times.argtypes = [vp, ctypes.POINTER(d), i]
    L.firm_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    for n in ("firm_pc_features", "firm_pc_net_input", "firm_pc_target", "firm_pc_axis", "firm_set_precond_table", "firm_pc_bin_volumes", "firm_pc_baseline",
              "firm_pc_residual_target", "firm_set_precond_residual"):
        getattr(L, n).argtypes = [vp, vp]
    L.firm_mlp_forward.argtypes = [vp, i, vp, vp, vp, vp]
    L.firm_mlp_to_bf16.argtypes = [vp, vp, vp]
    L.firm_mlp_forward_bf16.argtypes = [vp, vp, i, vp, vp, vp, vp]
    L.firm_mlp_grad.argtypes = [vp, i, vp, vp, vp, vp, vp, vp]
    L.firm_mlp_adam.argtypes = [vp, vp, vp, vp, i, ctypes.c_float, vp]
    L.firm_mlp_param_count.argtypes = []
    L.firm_mlp_work_floats.argtypes = [i]
    L.firm_mlp_work_floats.restype = ctypes.c_size_t
    L.firm_bin.argtypes = [vp, i, vp, i]
    L.firm_bin_info.argtypes = [vp] + [ctypes.POINTER(i)] * 5
    L.firm_batch_workspace_size.argtypes = [i, ctypes.POINTER(ctypes.c_size_t)]
    L.firm_batch_create.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(vp), i, vp, ctypes.c_size_t, vp]
    L.firm_batch_run.argtypes = [vp, ctypes.POINTER(firm_batch_item), i, i]
    L.firm_batch_solve.argtypes = [vp, ctypes.POINTER(firm_batch_item), i, d, i]
    L.firm_batch_set_network.argtypes = [vp, vp, vp]
    L.firm_batch_wait.argtypes = [vp, vp, vp]
    L.firm_batch_set_config.argtypes = [vp, i, i]
    L.firm_batch_get_config.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i)]
    L.firm_batch_tune.argtypes = [vp, ctypes.POINTER(firm_batch_item), i, i, ctypes.POINTER(d)]
    L.firm_batch_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    L.firm_batch_destroy.argtypes = [vp]
    L.firm_batch_destroy.restype = None
    L.firm_destroy.argtypes = [vp]
    L.firm_destroy.restype = None
    L.firm_strerror.argtypes = [i]
    L.firm_strerror.restype = ctypes.c_char_p
    for name in EXPORTED[:-2]:
        if name not in ("firm_mlp_work_floats", "firm_batch_destroy"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def strerror(code: int) -> str:
    return lib().firm_strerror(int(code)).decode()


def _ptr(a):
    """Raw address of a torch tensor / numpy array (None -> NULL).  Must be contiguous."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(f"unsupported array type {type(a)}")


def _check(code: int, what: str):
    if code != FIRM_OK:
        raise FirmError(code, what)


def make_params(N, M, n_groups=0, W=7, sigma=2.0, lam=0.0, lambda_mode=FIRM_LAMBDA_RELATIVE, disc_mode=0,
                img_dtype=FIRM_IMG_F32, flags=0) -> firm_params:
    return firm_params(N, M, n_groups, W, sigma, lam, lambda_mode, disc_mode, img_dtype, flags)


def make_groups(table) -> ctypes.Array | None:
    """(G, 6) table (defocus_A, kV, Cs_mm, amp_contrast, pixel_A, bfactor_A2) -> firm_ctf_group[G]."""
    table = np.asarray(table, float).reshape(-1, 6)
    if table.shape[0] == 0:
        return None
    arr = (firm_ctf_group * table.shape[0])()
    for g, row in enumerate(table):
        arr[g] = firm_ctf_group(*[float(v) for v in row])
    return arr


def firm_workspace_size(params: firm_params) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().firm_workspace_size(ctypes.byref(params), ctypes.byref(n)), "firm_workspace_size")
    return int(n.value)


def firm_plan(params: firm_params, groups, workspace, workspace_bytes: int, stream: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    g = ctypes.cast(groups, ctypes.POINTER(firm_ctf_group)) if groups is not None else None
    _check(lib().firm_plan(ctypes.byref(h), ctypes.byref(params), g, _ptr(workspace), workspace_bytes, stream),
           "firm_plan")
    return h


def firm_kernel(plan, M: int, R, group=None, khat_out=None):
    _check(lib().firm_kernel(plan, M, _ptr(R), _ptr(group), _ptr(khat_out)), "firm_kernel")


def firm_backproject(plan, M: int, images, shifts, R, group=None, rhs_out=None):
    _check(lib().firm_backproject(plan, M, _ptr(images), _ptr(shifts), _ptr(R), _ptr(group), _ptr(rhs_out)),
           "firm_backproject")


def firm_kernel_backproject(plan, M: int, images, shifts, R, group=None, khat_out=None, rhs_out=None):
    _check(lib().firm_kernel_backproject(plan, M, _ptr(images), _ptr(shifts), _ptr(R), _ptr(group), _ptr(khat_out),
                                         _ptr(rhs_out)), "firm_kernel_backproject")


def firm_load_sums(plan, ker_half=None, rhs=None):
    _check(lib().firm_load_sums(plan, _ptr(ker_half), _ptr(rhs)), "firm_load_sums")


def firm_stage_images(plan, M: int, images, staging, staging_bytes: int):
    _check(lib().firm_stage_images(plan, M, _ptr(images), _ptr(staging), int(staging_bytes)), "firm_stage_images")


def disc_size(N: int) -> int:
    """|K|, the number of integer frequencies with |k| <= N/2 (sizes the sample arrays)."""
    h = N // 2
    k = np.arange(-h, h + 1)
    return int(((k[:, None] ** 2 + k[None, :] ** 2) <= h * h).sum())


def firm_solve_nonneg(plan, x, max_iter: int, rel_tol: float, allow=()):
    """Returns (status, Toeplitz applies).  Raises unless the status is OK or in `allow`."""
    it = ctypes.c_int(0)
    st = lib().firm_solve_nonneg(plan, _ptr(x), int(max_iter), float(rel_tol), ctypes.byref(it))
    if st != FIRM_OK and st not in allow:
        _check(st, "firm_solve_nonneg")
    return st, it.value


def firm_set_damping(plan, mu: float):
    _check(lib().firm_set_damping(plan, float(mu)), "firm_set_damping")


def firm_forward(plan, M: int, V, R, group, out):
    _check(lib().firm_forward(plan, M, _ptr(V), _ptr(R), _ptr(group), _ptr(out)), "firm_forward")


def firm_data_residual(plan, M: int, V, images, shifts, R, group=None):
    """(sum |b - A V|^2, sum |b|^2) over every image's whole disc."""
    out = np.zeros(2, np.float64)
    _check(lib().firm_data_residual(plan, M, _ptr(V), _ptr(images), _ptr(shifts), _ptr(R), _ptr(group), _ptr(out)),
           "firm_data_residual")
    return float(out[0]), float(out[1])


def firm_cg_solve(plan, rhs, x, max_iter: int, rel_tol: float = 0.0, resid_hist=None, allow=()):
    """Returns (status, iterations).  Raises unless the status is OK or listed in `allow`."""
    it = ctypes.c_int(0)
    st = lib().firm_cg_solve(plan, _ptr(rhs), _ptr(x), int(max_iter), float(rel_tol), _ptr(resid_hist),
                             ctypes.byref(it))
    if st != FIRM_OK and st not in allow:
        raise FirmError(st, "firm_cg_solve")
    return st, int(it.value)


def firm_toeplitz_apply(plan, x, y):
    _check(lib().firm_toeplitz_apply(plan, _ptr(x), _ptr(y)), "firm_toeplitz_apply")


def firm_toeplitz_apply_static(N: int, khat, lam_eff: float, x, y, stream: int = 0):
    """y = Ker * x + lam_eff x without any device allocation (N <= 64; device arrays)."""
    _check(lib().firm_toeplitz_apply_static(int(N), _ptr(khat), float(lam_eff), _ptr(x), _ptr(y), stream),
           "firm_toeplitz_apply_static")


def firm_set_precond(plan, mode: int):
    _check(lib().firm_set_precond(plan, int(mode)), "firm_set_precond")


def firm_lambda_eff(plan) -> float:
    v = ctypes.c_double(0)
    _check(lib().firm_lambda_eff(plan, ctypes.byref(v)), "firm_lambda_eff")
    return float(v.value)


def firm_copy_out(plan, which: int, dst):
    _check(lib().firm_copy_out(plan, int(which), _ptr(dst)), "firm_copy_out")


def firm_set_timing(plan, on: bool):
    _check(lib().firm_set_timing(plan, 1 if on else 0), "firm_set_timing")


STAGES = ["bin_ker", "spread_ker", "fft_ker", "khat", "image_dft", "bin_rhs", "spread_rhs", "fft_rhs",
          "cg", "cg_iters", "gather_fused"]


def firm_stage_times(plan) -> dict:
    out = (ctypes.c_double * len(STAGES))()
    _check(lib().firm_stage_times(plan, out, len(STAGES)), "firm_stage_times")
    return dict(zip(STAGES, list(out)))


def firm_launch_count(plan) -> int:
    v = ctypes.c_longlong(0)
    _check(lib().firm_launch_count(plan, ctypes.byref(v)), "firm_launch_count")
    return int(v.value)


def firm_pc_features(plan, out):
    _check(lib().firm_pc_features(plan, _ptr(out)), "firm_pc_features")


def firm_pc_net_input(plan, out):
    _check(lib().firm_pc_net_input(plan, _ptr(out)), "firm_pc_net_input")


def firm_pc_target(plan, out):
    _check(lib().firm_pc_target(plan, _ptr(out)), "firm_pc_target")


def firm_pc_axis(plan):
    out = np.zeros(3, np.float32)
    _check(lib().firm_pc_axis(plan, out.ctypes.data), "firm_pc_axis")
    return out


def firm_set_precond_table(plan, table_log):
    _check(lib().firm_set_precond_table(plan, _ptr(table_log)), "firm_set_precond_table")


def firm_mlp_param_count() -> int:
    return int(lib().firm_mlp_param_count())


def firm_mlp_work_floats(batch: int) -> int:
    return int(lib().firm_mlp_work_floats(int(batch)))


def firm_mlp_forward(params, batch, x, y, work, stream=0):
    _check(lib().firm_mlp_forward(_ptr(params), int(batch), _ptr(x), _ptr(y), _ptr(work), stream), "firm_mlp_forward")


def firm_mlp_to_bf16(params, params_bf16, stream=0):
    _check(lib().firm_mlp_to_bf16(_ptr(params), _ptr(params_bf16), stream), "firm_mlp_to_bf16")


def firm_mlp_forward_bf16(params_bf16, params, batch, x, y, work, stream=0):
    _check(lib().firm_mlp_forward_bf16(_ptr(params_bf16), _ptr(params), int(batch), _ptr(x), _ptr(y), _ptr(work),
                                       stream), "firm_mlp_forward_bf16")


def firm_mlp_grad(params, batch, x, t, grad, work, loss, stream=0):
    _check(lib().firm_mlp_grad(_ptr(params), int(batch), _ptr(x), _ptr(t), _ptr(grad), _ptr(work), _ptr(loss), stream),
           "firm_mlp_grad")


def firm_mlp_adam(params, grad, m, v, step, lr, stream=0):
    _check(lib().firm_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(step), float(lr), stream),
           "firm_mlp_adam")


def firm_destroy(plan):
    if plan:
        lib().firm_destroy(plan)


# ---- batched reconstructions ----

def make_batch_items(items) -> ctypes.Array:
    """items: sequence of dicts with M, R, group, images, shifts, x (device tensors or None)."""
    arr = (firm_batch_item * len(items))()
    for k, it in enumerate(items):
        arr[k] = firm_batch_item(int(it["M"]), _ptr(it["R"]), _ptr(it.get("group")), _ptr(it["images"]),
                                 _ptr(it.get("shifts")), _ptr(it["x"]))
    return arr


def firm_batch_workspace_size(n_plans: int) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().firm_batch_workspace_size(int(n_plans), ctypes.byref(n)), "firm_batch_workspace_size")
    return int(n.value)


def firm_batch_create(plans, n_streams: int, workspace, workspace_bytes: int, stream: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    arr = (ctypes.c_void_p * len(plans))(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in plans])
    _check(lib().firm_batch_create(ctypes.byref(h), len(plans), arr, int(n_streams), _ptr(workspace),
                                   int(workspace_bytes), stream), "firm_batch_create")
    return h


def firm_batch_run(batch, items_arr, iters: int, flags: int):
    _check(lib().firm_batch_run(batch, items_arr, int(iters), int(flags)), "firm_batch_run")


def firm_batch_solve(batch, items_arr, max_iter: int, rel_tol: float, flags: int):
    _check(lib().firm_batch_solve(batch, items_arr, int(max_iter), float(rel_tol), int(flags)), "firm_batch_solve")


def firm_batch_set_network(batch, params_bf16, params):
    _check(lib().firm_batch_set_network(batch, _ptr(params_bf16), _ptr(params)), "firm_batch_set_network")


def firm_batch_wait(batch, n: int, allow=()):
    """Returns (status, per-plan statuses, per-plan iterations)."""
    st = np.zeros(n, np.int32)
    it = np.zeros(n, np.int32)
    r = lib().firm_batch_wait(batch, st.ctypes.data, it.ctypes.data)
    if r != FIRM_OK and r not in allow:
        raise FirmError(r, "firm_batch_wait")
    return r, st, it


def firm_batch_set_config(batch, n_streams: int, chunk: int):
    _check(lib().firm_batch_set_config(batch, int(n_streams), int(chunk)), "firm_batch_set_config")


def firm_batch_get_config(batch):
    a, b = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().firm_batch_get_config(batch, ctypes.byref(a), ctypes.byref(b)), "firm_batch_get_config")
    return int(a.value), int(b.value)


def firm_batch_tune(batch, items_arr, iters: int, flags: int) -> float:
    ms = ctypes.c_double(0)
    _check(lib().firm_batch_tune(batch, items_arr, int(iters), int(flags), ctypes.byref(ms)), "firm_batch_tune")
    return float(ms.value)


def firm_batch_launch_count(batch) -> int:
    v = ctypes.c_longlong(0)
    _check(lib().firm_batch_launch_count(batch, ctypes.byref(v)), "firm_batch_launch_count")
    return int(v.value)


def firm_batch_destroy(batch):
    if batch:
        lib().firm_batch_destroy(batch)


def firm_bin(plan, M: int, R, channel: int):
    _check(lib().firm_bin(plan, int(M), _ptr(R), int(channel)), "firm_bin")


def firm_bin_info(plan):
    """(n_work, n_points, bricks_per_axis, brick_depth, chunk) of the last firm_bin."""
    v = [ctypes.c_int(0) for _ in range(5)]
    _check(lib().firm_bin_info(plan, *[ctypes.byref(x) for x in v]), "firm_bin_info")
    return tuple(int(x.value) for x in v)


def firm_pc_bin_volumes(plan, out):
    _check(lib().firm_pc_bin_volumes(plan, _ptr(out)), "firm_pc_bin_volumes")


def firm_pc_baseline(plan, out):
    _check(lib().firm_pc_baseline(plan, _ptr(out)), "firm_pc_baseline")


def firm_pc_residual_target(plan, out):
    _check(lib().firm_pc_residual_target(plan, _ptr(out)), "firm_pc_residual_target")


def firm_set_precond_residual(plan, delta):
    _check(lib().firm_set_precond_residual(plan, _ptr(delta)), "firm_set_precond_residual")
