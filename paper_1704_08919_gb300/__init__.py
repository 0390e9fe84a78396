"""GPU scoring of candidate laser pulses by the electron-positron pair number
(arXiv 1704.08919): a thin ctypes binding over the C ABI of libpp
(include/pp.h).  The functions take and return torch CUDA tensors and only
marshal arguments; every step of the computation runs in the library's CUDA
kernels.  There is no CPU fallback: calling any function without the built
library raises.

    A, E, s = synth_field(params, spec)                  # Sec. III pulse model
    N, n    = pair_number(A, dt, grid, precision="fp32")  # Sec. II.A + Eq. (opt_prob)
    trial   = de_propose(pop, lo, hi, periodic, F, CR, seed, gen)   # Sec. IV.B
    de_select(pop, fit, trial, trial_fit)
    de_step(pop, fit, spec, grid, lo, hi, periodic, F, CR, seed, gen)
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpp.so")

PP_OK = 0
PP_ERR_INVALID_ARG = 1
PP_ERR_CUDA = 2
PP_ERR_NONFINITE = 3
PP_ERR_DEGENERATE_FIELD = 4
PP_ERR_TIMEOUT = 5
PP_ERR_NOT_IMPLEMENTED = 6

PP_FP64 = 0
PP_FP32 = 1
PP_FP32_FAST = 2
PRECISIONS = {"fp64": PP_FP64, "fp32": PP_FP32, "fp32fast": PP_FP32_FAST, PP_FP64: PP_FP64,
              PP_FP32: PP_FP32, PP_FP32_FAST: PP_FP32_FAST}

PP_RK4 = 0
PP_MAGNUS4 = 1
PP_SPLIT2 = 2
SCHEMES = {"rk4": PP_RK4, "magnus4": PP_MAGNUS4, "split2": PP_SPLIT2,
           PP_RK4: PP_RK4, PP_MAGNUS4: PP_MAGNUS4, PP_SPLIT2: PP_SPLIT2}

EXPORTS = ("pp_synth_field", "pp_pair_number", "pp_de_propose", "pp_de_select", "pp_de_step",
           "pp_sync_status", "pp_set_wait_limit", "pp_set_skip_copies", "pp_last_error",
           "pp_version", "pp_profile_begin", "pp_profile_end", "pp_tune_pair_number",
           "pp_num_launch_configs", "pp_launch_config", "pp_clear_tuning", "pp_pair_number_static",
           "pp_static_scratch_bytes", "pp_batch_create", "pp_batch_destroy", "pp_batch_info",
           "pp_batch_synth", "pp_batch_pair_number", "pp_batch_tune", "pp_batch_set_generation",
           "pp_batch_de_step", "pp_batch_de_run", "pp_packed_bf16_bytes", "pp_pack_bf16",
           "pp_gemm_bf16", "pp_mlp_create", "pp_mlp_destroy", "pp_mlp_num_params",
           "pp_mlp_set_params", "pp_mlp_get_params", "pp_mlp_forward", "pp_mlp_loss_grad",
           "pp_mlp_train_step", "pp_mlp_features", "pp_de_screened_step", "pp_mlp_fit",
           "pp_mlp_log_targets", "pp_mlp_init", "pp_al_search", "pp_synth_field_raw",
           "pp_synth_vjp", "pp_qke_pair_number", "pp_qke_sample_gradient", "pp_qke_gradient",
           "pp_local_search", "pp_release_scratch", "pp_pair_number_grids",
           "pp_set_qke_state_budget", "pp_fma_rate")


class ALOptions(ctypes.Structure):
    """pp_al_options."""
    _fields_ = [("mu0", ctypes.c_double), ("xi", ctypes.c_double), ("outer", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("gtol", ctypes.c_double), ("ctol", ctypes.c_double)]


ObjectiveFn = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int32,
                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double))


class PPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libpp error %d: %s" % (code, msg))
        self.code = code


class FieldSpec(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("order", ctypes.c_int32), ("w_min", ctypes.c_double),
                ("w_max", ctypes.c_double), ("T", ctypes.c_double), ("fluence", ctypes.c_double),
                ("n_steps", ctypes.c_int32), ("envelope", ctypes.c_int32)]


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double),
                ("y1", ctypes.c_double), ("z0", ctypes.c_double), ("z1", ctypes.c_double),
                ("mirror_z", ctypes.c_int32)]


_lib = None
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_d = ctypes.c_double
_u64 = ctypes.c_uint64


def lib():
    """The loaded libpp.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libpp.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        L.pp_synth_field.argtypes = [_vp, _i32, ctypes.POINTER(FieldSpec), _vp, _i32, _vp, _vp, _vp]
        L.pp_pair_number.argtypes = [_vp, _i32, _i32, _vp, _d, ctypes.POINTER(Grid), _i32, _i32,
                                     _vp, _vp, _vp]
        L.pp_de_propose.argtypes = [_vp, _i32, _i32, _vp, _vp, _vp, _d, _d, _u64, _u64, _vp, _vp]
        L.pp_de_select.argtypes = [_vp, _vp, _vp, _vp, _i32, _i32, _vp]
        L.pp_de_step.argtypes = [_vp, _vp, _i32, ctypes.POINTER(FieldSpec), ctypes.POINTER(Grid),
                                 _i32, _i32, _vp, _vp, _vp, _d, _d, _u64, _u64, _vp, _vp, _vp]
        L.pp_sync_status.argtypes = [_vp]
        L.pp_set_wait_limit.argtypes = [ctypes.c_int64]
        L.pp_set_wait_limit.restype = ctypes.c_int64
        L.pp_set_qke_state_budget.argtypes = [ctypes.c_int64]
        L.pp_set_qke_state_budget.restype = ctypes.c_int64
        L.pp_fma_rate.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
        L.pp_set_skip_copies.argtypes = [ctypes.c_int]
        L.pp_last_error.restype = ctypes.c_char_p
        L.pp_profile_end.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
        L.pp_tune_pair_number.argtypes = [_vp, _i32, _i32, _vp, _d, ctypes.POINTER(Grid), _i32,
                                          _i32, _vp, ctypes.POINTER(_i32),
                                          ctypes.POINTER(ctypes.c_float), _vp]
        L.pp_launch_config.argtypes = [_i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]
        L.pp_clear_tuning.restype = None
        L.pp_pair_number_static.argtypes = L.pp_pair_number.argtypes
        L.pp_pair_number_grids.argtypes = [_vp, _i32, _i32, _vp, _d, _vp, _i32, _i32, _i32, _vp, _vp, _vp]
        L.pp_static_scratch_bytes.restype = ctypes.c_size_t
        L.pp_batch_create.argtypes = [_i32, ctypes.POINTER(FieldSpec), ctypes.POINTER(Grid), _i32,
                                      _i32, _d, ctypes.POINTER(_vp)]
        L.pp_batch_destroy.argtypes = [_vp]
        L.pp_batch_destroy.restype = None
        L.pp_batch_info.argtypes = [_vp, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(_i32)]
        L.pp_batch_synth.argtypes = [_vp, _vp, _vp, _vp]
        L.pp_batch_pair_number.argtypes = [_vp, _vp, _vp, _vp, _vp]
        L.pp_batch_tune.argtypes = [_vp, _vp, _vp, ctypes.POINTER(_i32),
                                    ctypes.POINTER(ctypes.c_float), _vp]
        L.pp_batch_set_generation.argtypes = [_vp, _u64, _vp]
        L.pp_batch_de_step.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _d, _d, _u64, _vp]
        L.pp_packed_bf16_bytes.argtypes = [_i32, _i32]
        L.pp_packed_bf16_bytes.restype = ctypes.c_size_t
        L.pp_pack_bf16.argtypes = [_vp, _i32, _i32, _i32, _i32, _vp, _vp]
        L.pp_gemm_bf16.argtypes = [_vp, _vp, _vp, _i32, _i32, _i32, _i32, _vp]
        L.pp_mlp_create.argtypes = [_i32, _i32, _i32, ctypes.POINTER(_vp)]
        L.pp_mlp_destroy.argtypes = [_vp]
        L.pp_mlp_destroy.restype = None
        L.pp_mlp_num_params.argtypes = [_vp]
        L.pp_mlp_num_params.restype = ctypes.c_int64
        L.pp_mlp_set_params.argtypes = [_vp, _vp, _vp]
        L.pp_mlp_get_params.argtypes = [_vp, _vp, _vp]
        L.pp_mlp_forward.argtypes = [_vp, _vp, _i32, _vp, _vp]
        L.pp_mlp_loss_grad.argtypes = [_vp, _vp, _vp, _i32, _vp, _vp, _vp]
        L.pp_mlp_train_step.argtypes = [_vp, _vp, _vp, _i32, ctypes.c_float, _vp, _vp]
        L.pp_mlp_features.argtypes = [_vp, _i32, _i32, _vp, _vp, _vp, _vp]
        L.pp_de_screened_step.argtypes = [_vp, _vp, _i32, ctypes.POINTER(FieldSpec),
                                          ctypes.POINTER(Grid), _i32, _i32, _vp, _vp, _vp, _d, _d,
                                          _u64, _u64, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp]
        L.pp_mlp_fit.argtypes = [_vp, _vp, _vp, _i32, _i32, _i32, ctypes.c_float, ctypes.c_float,
                                 ctypes.c_uint64, _vp, _vp]
        L.pp_mlp_log_targets.argtypes = [_vp, _i32, _d, _d, _d, _vp, _vp]
        L.pp_mlp_init.argtypes = [_vp, _u64, _vp]
        L.pp_synth_field_raw.argtypes = [_vp, _i32, ctypes.POINTER(FieldSpec), _vp, _vp, _vp, _i32,
                                         _vp, _vp]
        L.pp_synth_vjp.argtypes = [_vp, _i32, ctypes.POINTER(FieldSpec), _vp, _i32, _vp, _vp, _vp,
                                   _vp]
        L.pp_qke_pair_number.argtypes = [_vp, _vp, _vp, _i32, _i32, _i32, _d, ctypes.POINTER(Grid),
                                         _i32, _vp, _vp, _vp]
        L.pp_qke_sample_gradient.argtypes = [_vp, _vp, _vp, _i32, _i32, _i32, _d,
                                             ctypes.POINTER(Grid), _i32, _vp, _vp, _i32, _vp]
        L.pp_qke_gradient.argtypes = [_vp, _i32, ctypes.POINTER(FieldSpec), ctypes.POINTER(Grid),
                                      _i32, _vp, _vp, _vp, _vp, _vp]
        L.pp_local_search.argtypes = [_vp, _i32, ctypes.POINTER(FieldSpec), ctypes.POINTER(Grid),
                                      _i32, _d, ctypes.POINTER(ALOptions), _vp, _vp, _vp, _vp, _vp,
                                      _vp, _vp]
        L.pp_al_search.argtypes = [_i32, _i32, _vp, ObjectiveFn, _vp, ctypes.POINTER(ALOptions),
                                   _vp, _vp, _vp, _vp, _vp, _vp]
        L.pp_batch_de_run.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _d, _d, _u64, _i32, _vp]
        _lib = L
    return _lib


def _check(rc):
    if rc != PP_OK:
        raise PPError(rc, lib().pp_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def field_spec(K, order, w_min, w_max, T, fluence, n_steps, envelope=0):
    return FieldSpec(K, order, w_min, w_max, T, fluence, n_steps, envelope)


def _spec(spec):
    if isinstance(spec, FieldSpec):
        return spec
    return FieldSpec(spec["K"], spec["order"], spec["w_min"], spec["w_max"], spec["T"],
                     spec["fluence"], spec["n_steps"], spec.get("envelope", 0))


def _grid(grid):
    if isinstance(grid, Grid):
        return grid
    return Grid(grid["nx"], grid["ny"], grid["nz"], grid["x0"], grid["x1"], grid["y0"], grid["y1"],
                grid["z0"], grid["z1"], int(grid.get("mirror_z", 0)))


def synth_field(params, spec, want_E=False, want_scale=False, stream=None, out=None):
    """pp_synth_field: params [ncand, 4K] float64 CUDA -> A [ncand, 2, 2n+1] (and E, scale)."""
    import torch
    sp = _spec(spec)
    ncand = params.shape[0]
    ld = 2 * sp.n_steps + 1
    dev = params.device
    A = out if out is not None else torch.empty((ncand, 2, ld), dtype=torch.float64, device=dev)
    E = torch.empty_like(A) if want_E else None
    s = torch.empty(ncand, dtype=torch.float64, device=dev) if want_scale else None
    _check(lib().pp_synth_field(_ptr(params), ncand, ctypes.byref(sp), _ptr(A), A.shape[-1],
                                _ptr(E), _ptr(s), _stream(stream)))
    return A, E, s


def pair_number(A, dt, grid, precision="fp32", n_steps=None, want_n=False, stream=None, N_out=None,
                scheme="rk4"):
    """pp_pair_number: A [ncand, 2, ld] float64 CUDA -> N [ncand] (and n [ncand, nz, ny, nx])."""
    import torch
    g = _grid(grid)
    ncand, _, ld = A.shape
    N = N_out if N_out is not None else torch.empty(ncand, dtype=torch.float64, device=A.device)
    n = (torch.empty((ncand, g.nz, g.ny, g.nx), dtype=torch.float64, device=A.device)
         if want_n else None)
    ns = None
    if n_steps is not None:
        arr = (ctypes.c_int32 * ncand)(*[int(x) for x in n_steps])
        ns = ctypes.cast(arr, ctypes.c_void_p)
    _check(lib().pp_pair_number(_ptr(A), ncand, ld, ns, float(dt), ctypes.byref(g),
                                PRECISIONS[precision], SCHEMES[scheme], _ptr(N), _ptr(n),
                                _stream(stream)))
    return N, n


def pair_number_static(A, dt, grid, precision="fp32", n_steps=None, want_n=False, stream=None,
                       N_out=None, scheme="rk4"):
    """pp_pair_number_static: pair_number with no device allocation (fixed static scratch)."""
    import torch
    g = _grid(grid)
    ncand, _, ld = A.shape
    N = N_out if N_out is not None else torch.empty(ncand, dtype=torch.float64, device=A.device)
    n = (torch.empty((ncand, g.nz, g.ny, g.nx), dtype=torch.float64, device=A.device)
         if want_n else None)
    ns = None
    if n_steps is not None:
        arr = (ctypes.c_int32 * ncand)(*[int(x) for x in n_steps])
        ns = ctypes.cast(arr, ctypes.c_void_p)
    _check(lib().pp_pair_number_static(_ptr(A), ncand, ld, ns, float(dt), ctypes.byref(g),
                                       PRECISIONS[precision], SCHEMES[scheme], _ptr(N), _ptr(n),
                                       _stream(stream)))
    return N, n


def pair_number_grids(A, dt, grids, precision="fp32", n_steps=None, want_n=False, stream=None, scheme="rk4"):
    """pp_pair_number_grids: A [ncand, 2, ld] float64 CUDA and a grid per candidate (or one) ->
    N [ncand] (and n, the candidates' n(p) concatenated, 1-D)."""
    import torch
    gs = [_grid(g) for g in grids]
    ncand, _, ld = A.shape
    arr = (Grid * len(gs))(*gs)
    N = torch.empty(ncand, dtype=torch.float64, device=A.device)
    nmodes = [g.nx * g.ny * g.nz for g in gs] if len(gs) == ncand else [gs[0].nx * gs[0].ny * gs[0].nz] * ncand
    n = torch.empty(sum(nmodes), dtype=torch.float64, device=A.device) if want_n else None
    ns = None
    if n_steps is not None:
        nsa = (ctypes.c_int32 * ncand)(*[int(x) for x in n_steps])
        ns = ctypes.cast(nsa, ctypes.c_void_p)
    _check(lib().pp_pair_number_grids(_ptr(A), ncand, ld, ns, float(dt), ctypes.cast(arr, ctypes.c_void_p),
                                      len(gs), PRECISIONS[precision], SCHEMES[scheme], _ptr(N), _ptr(n),
                                      _stream(stream)))
    return N, n


def tune_pair_number(A, dt, grid, precision="fp32", scheme="magnus4", n_steps=None, stream=None):
    """pp_tune_pair_number: time every launch configuration on these inputs, remember the
    fastest for this workload shape.  Returns (chosen index, per-configuration ms, N)."""
    import torch
    g = _grid(grid)
    ncand, _, ld = A.shape
    N = torch.empty(ncand, dtype=torch.float64, device=A.device)
    nc = lib().pp_num_launch_configs()
    ms = (ctypes.c_float * nc)()
    chosen = _i32(-1)
    ns = None
    if n_steps is not None:
        arr = (ctypes.c_int32 * ncand)(*[int(x) for x in n_steps])
        ns = ctypes.cast(arr, ctypes.c_void_p)
    _check(lib().pp_tune_pair_number(_ptr(A), ncand, ld, ns, float(dt), ctypes.byref(g),
                                     PRECISIONS[precision], SCHEMES[scheme], _ptr(N),
                                     ctypes.byref(chosen), ms, _stream(stream)))
    return chosen.value, list(ms), N


def launch_configs():
    """[(threads per CTA, tile bytes)] of the propagation kernel's launch configurations."""
    out = []
    for k in range(lib().pp_num_launch_configs()):
        t, b = _i32(0), _i32(0)
        _check(lib().pp_launch_config(k, ctypes.byref(t), ctypes.byref(b)))
        out.append((t.value, b.value))
    return out


def clear_tuning():
    lib().pp_clear_tuning()


def pack_bf16(X, transpose=False, stream=None):
    """pp_pack_bf16: FP32 CUDA matrix -> packed BF16 tile layout (uint8 tensor).
    With transpose=True, X (cols x rows) is packed as its transpose (rows x cols)."""
    import torch
    rows, cols = (X.shape[1], X.shape[0]) if transpose else (X.shape[0], X.shape[1])
    P = torch.empty(lib().pp_packed_bf16_bytes(rows, cols), dtype=torch.uint8, device=X.device)
    _check(lib().pp_pack_bf16(_ptr(X), rows, cols, X.stride(0), int(transpose), _ptr(P),
                              _stream(stream)))
    return P, rows, cols


def gemm_bf16(Ap, Bp, M, N, K, out=None, stream=None):
    """pp_gemm_bf16: D[M][N] = A . B^T from packed BF16 operands (FP32 result)."""
    import torch
    D = out if out is not None else torch.empty((M, N), dtype=torch.float32, device=Ap.device)
    _check(lib().pp_gemm_bf16(_ptr(Ap), _ptr(Bp), _ptr(D), M, N, K, D.stride(0), _stream(stream)))
    return D


class Surrogate:
    """pp_mlp_*: the surrogate network (d_in -> H -> H -> H -> 1, GELU)."""

    def __init__(self, d_in, hidden=256, max_batch=4096):
        h = _vp()
        _check(lib().pp_mlp_create(int(d_in), int(hidden), int(max_batch), ctypes.byref(h)))
        self.h = h
        self.d_in, self.hidden, self.max_batch = d_in, hidden, max_batch
        self.nparam = lib().pp_mlp_num_params(h)

    def close(self):
        if self.h:
            lib().pp_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params, stream=None):
        """params: FP32 CUDA tensor [n_params]."""
        _check(lib().pp_mlp_set_params(self.h, _ptr(params), _stream(stream)))

    def init(self, seed, stream=None):
        """pp_mlp_init: He initialisation from a counter-based generator."""
        _check(lib().pp_mlp_init(self.h, int(seed), _stream(stream)))

    def get_params(self, stream=None):
        import torch
        out = torch.empty(self.nparam, dtype=torch.float32, device="cuda")
        _check(lib().pp_mlp_get_params(self.h, _ptr(out), _stream(stream)))
        return out

    def forward(self, X, stream=None):
        import torch
        y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        _check(lib().pp_mlp_forward(self.h, _ptr(X), X.shape[0], _ptr(y), _stream(stream)))
        return y

    def loss_grad(self, X, t, stream=None):
        import torch
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        g = torch.empty(self.nparam, dtype=torch.float32, device=X.device)
        _check(lib().pp_mlp_loss_grad(self.h, _ptr(X), _ptr(t), X.shape[0], _ptr(loss), _ptr(g),
                                      _stream(stream)))
        return loss, g

    def train_step(self, X, t, lr, stream=None):
        import torch
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        _check(lib().pp_mlp_train_step(self.h, _ptr(X), _ptr(t), X.shape[0], float(lr), _ptr(loss),
                                       _stream(stream)))
        return loss

    def fit(self, X, t, batch, epochs, lr0, lr1, seed=0, stream=None):
        """pp_mlp_fit; seed 0 keeps the row order, others shuffle it per epoch.  Returns
        the loss of each epoch's last slice (FP32 CUDA tensor)."""
        import torch
        loss = torch.empty(epochs, dtype=torch.float32, device=X.device)
        _check(lib().pp_mlp_fit(self.h, _ptr(X), _ptr(t), X.shape[0], int(batch), int(epochs),
                                float(lr0), float(lr1), int(seed), _ptr(loss), _stream(stream)))
        return loss


def log_targets(N, floor, shift, scale, stream=None):
    """pp_mlp_log_targets: (log10(max(N, floor)) - shift) / scale as FP32."""
    import torch
    t = torch.empty(N.shape[0], dtype=torch.float32, device=N.device)
    _check(lib().pp_mlp_log_targets(_ptr(N), N.shape[0], float(floor), float(shift), float(scale),
                                    _ptr(t), _stream(stream)))
    return t


SCREEN_MODES = {"individual": 0, "global": 1}


def de_screened_step(pop, fit, spec, grid, lo, hi, periodic, F, CR, seed, generation, R, net,
                     precision="fp32fast", scheme="magnus4", mode="individual", trial_out=None,
                     trial_fit_out=None, pred_out=None, kept_out=None, stream=None):
    """pp_de_screened_step: R proposals per individual, the network keeps NP, exact scoring."""
    sp, g = _spec(spec), _grid(grid)
    _check(lib().pp_de_screened_step(_ptr(pop), _ptr(fit), pop.shape[0], ctypes.byref(sp),
                                     ctypes.byref(g), PRECISIONS[precision], SCHEMES[scheme],
                                     _ptr(lo), _ptr(hi), _ptr(periodic), float(F), float(CR),
                                     int(seed), int(generation), int(R), SCREEN_MODES[mode], net.h,
                                     _ptr(trial_out), _ptr(trial_fit_out), _ptr(pred_out),
                                     _ptr(kept_out), _stream(stream)))


def mlp_features(params, lo, hi, stream=None):
    """pp_mlp_features: FP64 parameter vectors -> normalised FP32 network inputs."""
    import torch
    B, D = params.shape
    X = torch.empty((B, D), dtype=torch.float32, device=params.device)
    _check(lib().pp_mlp_features(_ptr(params), B, D, _ptr(lo), _ptr(hi), _ptr(X), _stream(stream)))
    return X


class Batch:
    """pp_batch_*: slots with their own pulse length, step count and momentum grid."""

    def __init__(self, specs, grids, dt, precision="fp32", scheme="magnus4"):
        n = len(specs)
        sp = (FieldSpec * n)(*[_spec(x) for x in specs])
        gr = (Grid * n)(*[_grid(x) for x in grids])
        h = _vp()
        _check(lib().pp_batch_create(n, sp, gr, PRECISIONS[precision], SCHEMES[scheme], float(dt),
                                     ctypes.byref(h)))
        self.h = h
        self.ncand = n
        self.grids = [_grid(x) for x in grids]
        ld, tm, cfg = _i32(0), ctypes.c_int64(0), _i32(0)
        _check(lib().pp_batch_info(h, ctypes.byref(ld), ctypes.byref(tm), ctypes.byref(cfg)))
        self.ld, self.total_modes = ld.value, tm.value

    def close(self):
        if self.h:
            lib().pp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def config(self):
        cfg = _i32(0)
        _check(lib().pp_batch_info(self.h, None, None, ctypes.byref(cfg)))
        return cfg.value

    def synth(self, params, stream=None):
        import torch
        A = torch.zeros((self.ncand, 2, self.ld), dtype=torch.float64, device=params.device)
        _check(lib().pp_batch_synth(self.h, _ptr(params), _ptr(A), _stream(stream)))
        return A

    def pair_number(self, A, want_n=False, stream=None):
        import torch
        N = torch.empty(self.ncand, dtype=torch.float64, device=A.device)
        n = (torch.empty(self.total_modes, dtype=torch.float64, device=A.device) if want_n else None)
        _check(lib().pp_batch_pair_number(self.h, _ptr(A), _ptr(N), _ptr(n), _stream(stream)))
        return N, n

    def tune(self, A, stream=None):
        import torch
        N = torch.empty(self.ncand, dtype=torch.float64, device=A.device)
        ms = (ctypes.c_float * 6)()
        chosen = _i32(-1)
        _check(lib().pp_batch_tune(self.h, _ptr(A), _ptr(N), ctypes.byref(chosen), ms,
                                   _stream(stream)))
        return chosen.value, list(ms)

    def set_generation(self, generation, stream=None):
        _check(lib().pp_batch_set_generation(self.h, int(generation), _stream(stream)))

    def de_step(self, pop, fit, lo, hi, periodic, F, CR, seed, stream=None):
        _check(lib().pp_batch_de_step(self.h, _ptr(pop), _ptr(fit), _ptr(lo), _ptr(hi),
                                      _ptr(periodic), float(F), float(CR), int(seed),
                                      _stream(stream)))

    def de_run(self, pop, fit, lo, hi, periodic, F, CR, seed, generations, stream=None):
        _check(lib().pp_batch_de_run(self.h, _ptr(pop), _ptr(fit), _ptr(lo), _ptr(hi),
                                     _ptr(periodic), float(F), float(CR), int(seed),
                                     int(generations), _stream(stream)))


def de_propose(pop, lo, hi, periodic, F, CR, seed, generation, stream=None, out=None):
    """pp_de_propose: DE/rand/1/bin trial vectors."""
    import torch
    NP, D = pop.shape
    trial = out if out is not None else torch.empty_like(pop)
    _check(lib().pp_de_propose(_ptr(pop), NP, D, _ptr(lo), _ptr(hi), _ptr(periodic), float(F),
                               float(CR), int(seed), int(generation), _ptr(trial), _stream(stream)))
    return trial


def de_select(pop, fit, trial, trial_fit, stream=None):
    """pp_de_select: greedy selection (maximisation), in place."""
    NP, D = pop.shape
    _check(lib().pp_de_select(_ptr(pop), _ptr(fit), _ptr(trial), _ptr(trial_fit), NP, D,
                              _stream(stream)))


def de_step(pop, fit, spec, grid, lo, hi, periodic, F, CR, seed, generation, precision="fp32",
            trial_out=None, trial_fit_out=None, stream=None, scheme="rk4"):
    """pp_de_step: one DE generation (propose, synthesise, score, select) in place."""
    sp, g = _spec(spec), _grid(grid)
    NP = pop.shape[0]
    _check(lib().pp_de_step(_ptr(pop), _ptr(fit), NP, ctypes.byref(sp), ctypes.byref(g),
                            PRECISIONS[precision], SCHEMES[scheme], _ptr(lo), _ptr(hi),
                            _ptr(periodic), float(F),
                            float(CR), int(seed), int(generation), _ptr(trial_out),
                            _ptr(trial_fit_out), _stream(stream)))


def sync_status(stream=None):
    """pp_sync_status: wait for the stream; return (and clear) the device status code."""
    return lib().pp_sync_status(_stream(stream))


def release_scratch():
    """pp_release_scratch: free the library's scratch on the current device."""
    _check(lib().pp_release_scratch())


def profile_begin():
    """pp_profile_begin: start timing every propagation-kernel launch with CUDA events."""
    _check(lib().pp_profile_begin())


def profile_end():
    """pp_profile_end: (total kernel milliseconds, launches) since profile_begin()."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    _check(lib().pp_profile_end(ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def set_wait_limit(limit):
    return lib().pp_set_wait_limit(int(limit))


def set_skip_copies(skip):
    return lib().pp_set_skip_copies(int(skip))


def fma_rate(precision="fp32", stream=None):
    """pp_fma_rate: the FMA rate this GPU sustains in flop/s (the roofline denominator)."""
    out = ctypes.c_double(0.0)
    _check(lib().pp_fma_rate(PRECISIONS[precision], ctypes.byref(out), _stream(stream)))
    return out.value


def set_qke_state_budget(nbytes):
    """pp_set_qke_state_budget: device bytes the QKE adjoint may keep for forward states
    (negative: the default, half the device's memory).  Returns the previous setting
    (-1: the default)."""
    return lib().pp_set_qke_state_budget(int(nbytes))


def al_search(x0, fn, mu0=1.0, xi=0.5, outer=10, max_iter=200, gtol=1e-6, ctol=1e-8):
    """pp_al_search with a Python objective fn(X[count, n]) -> (J, gJ, C, gC) (numpy).

    Returns dict(x, J, C, lam, evals, outer, status) with one row / entry per start."""
    import numpy as np
    x = np.array(x0, dtype=np.float64, copy=True, ndmin=2)
    nstart, n = x.shape
    err = []

    def cb(ctx, count, xp, Jp, gJp, Cp, gCp):
        try:
            X = np.ctypeslib.as_array(xp, shape=(count, n)).copy()
            J, gJ, C, gC = fn(X)
            np.ctypeslib.as_array(Jp, shape=(count,))[:] = J
            np.ctypeslib.as_array(gJp, shape=(count, n))[:] = gJ
            np.ctypeslib.as_array(Cp, shape=(count,))[:] = C
            np.ctypeslib.as_array(gCp, shape=(count, n))[:] = gC
            return 0
        except Exception as e:  # noqa: BLE001 -- reported after the search returns
            err.append(e)
            return PP_ERR_INVALID_ARG
    opt = ALOptions(mu0, xi, outer, max_iter, gtol, ctol)
    J, C, lam = np.zeros(nstart), np.zeros(nstart), np.zeros(nstart)
    ev, ou, stt = (np.zeros(nstart, dtype=np.int32) for _ in range(3))
    f = ObjectiveFn(cb)
    rc = lib().pp_al_search(n, nstart, x.ctypes.data, f, None, ctypes.byref(opt), J.ctypes.data,
                            C.ctypes.data, lam.ctypes.data, ev.ctypes.data, ou.ctypes.data,
                            stt.ctypes.data)
    if err:
        raise err[0]
    _check(rc)
    return dict(x=x, J=J, C=C, lam=lam, evals=ev, outer=ou, status=stt)


# ----------------------------------------------------------------------------- QKE local search


def synth_field_raw(params, spec, stream=None):
    """pp_synth_field_raw: (A, E, Ed [ncand, 2, 2n+1], U [ncand]) without renormalisation."""
    import torch
    sp = _spec(dict(spec, fluence=spec.get("fluence", 1.0)))
    ncand, ld = params.shape[0], 2 * sp.n_steps + 1
    A, E, Ed = (torch.empty((ncand, 2, ld), dtype=torch.float64, device=params.device)
                for _ in range(3))
    U = torch.empty(ncand, dtype=torch.float64, device=params.device)
    _check(lib().pp_synth_field_raw(_ptr(params), ncand, ctypes.byref(sp), _ptr(A), _ptr(E),
                                    _ptr(Ed), ld, _ptr(U), _stream(stream)))
    return A, E, Ed, U


def synth_vjp(params, spec, g, stream=None):
    """pp_synth_vjp: g [ncand, 6, ldg] = dJ/d(samples) -> (grad [ncand, 4K], U, dU)."""
    import torch
    sp = _spec(dict(spec, fluence=spec.get("fluence", 1.0)))
    ncand = params.shape[0]
    grad, dU = (torch.empty((ncand, 4 * sp.K), dtype=torch.float64, device=params.device)
                for _ in range(2))
    U = torch.empty(ncand, dtype=torch.float64, device=params.device)
    _check(lib().pp_synth_vjp(_ptr(params), ncand, ctypes.byref(sp), _ptr(g), g.shape[-1],
                              _ptr(grad), _ptr(U), _ptr(dU), _stream(stream)))
    return grad, U, dU


def qke_pair_number(A, E, Ed, dt, grid, precision="fp64", n_steps=None, want_n=False, stream=None):
    """pp_qke_pair_number: J [ncand] (and f [ncand, nz, ny, nx])."""
    import torch
    g = _grid(grid)
    ncand, _, ld = A.shape
    ns = n_steps if n_steps is not None else (ld - 1) // 2
    J = torch.empty(ncand, dtype=torch.float64, device=A.device)
    n = (torch.empty((ncand, g.nz, g.ny, g.nx), dtype=torch.float64, device=A.device)
         if want_n else None)
    _check(lib().pp_qke_pair_number(_ptr(A), _ptr(E), _ptr(Ed), ncand, ld, ns, float(dt),
                                    ctypes.byref(g), PRECISIONS[precision], _ptr(J), _ptr(n),
                                    _stream(stream)))
    return J, n


def qke_sample_gradient(A, E, Ed, dt, grid, precision="fp64", n_steps=None, stream=None):
    """pp_qke_sample_gradient: (J [ncand], g [ncand, 6, 2n+1]) with g = dJ/d(samples)."""
    import torch
    gr = _grid(grid)
    ncand, _, ld = A.shape
    ns = n_steps if n_steps is not None else (ld - 1) // 2
    J = torch.empty(ncand, dtype=torch.float64, device=A.device)
    g = torch.empty((ncand, 6, 2 * ns + 1), dtype=torch.float64, device=A.device)
    _check(lib().pp_qke_sample_gradient(_ptr(A), _ptr(E), _ptr(Ed), ncand, ld, ns, float(dt),
                                        ctypes.byref(gr), PRECISIONS[precision], _ptr(J), _ptr(g),
                                        g.shape[-1], _stream(stream)))
    return J, g


def qke_gradient(params, spec, grid, precision="fp64", want_grad=True, stream=None):
    """pp_qke_gradient: (J, gJ, U, dU) for params [ncand, 4K] (gJ None unless want_grad)."""
    import torch
    sp = _spec(dict(spec, fluence=spec.get("fluence", 1.0)))
    ncand = params.shape[0]
    J, U = (torch.empty(ncand, dtype=torch.float64, device=params.device) for _ in range(2))
    gJ = (torch.empty((ncand, 4 * sp.K), dtype=torch.float64, device=params.device)
          if want_grad else None)
    dU = torch.empty((ncand, 4 * sp.K), dtype=torch.float64, device=params.device)
    _check(lib().pp_qke_gradient(_ptr(params), ncand, ctypes.byref(sp), ctypes.byref(_grid(grid)),
                                 PRECISIONS[precision], _ptr(J), _ptr(gJ), _ptr(U), _ptr(dU),
                                 _stream(stream)))
    return J, gJ, U, dU


def local_search(x0, spec, grid, U_const, precision="fp64", mu0=1.0, xi=0.5, outer=10,
                 max_iter=200, gtol=1e-6, ctol=1e-8, stream=None):
    """pp_local_search from host starts x0 [nstart, 4K]; returns dict like al_search."""
    import numpy as np
    x = np.array(x0, dtype=np.float64, copy=True, ndmin=2)
    nstart = x.shape[0]
    sp = _spec(dict(spec, fluence=spec.get("fluence", 1.0)))
    opt = ALOptions(mu0, xi, outer, max_iter, gtol, ctol)
    J, C, lam = np.zeros(nstart), np.zeros(nstart), np.zeros(nstart)
    ev, ou, stt = (np.zeros(nstart, dtype=np.int32) for _ in range(3))
    _check(lib().pp_local_search(x.ctypes.data, nstart, ctypes.byref(sp), ctypes.byref(_grid(grid)),
                                 PRECISIONS[precision], float(U_const), ctypes.byref(opt),
                                 J.ctypes.data, C.ctypes.data, lam.ctypes.data, ev.ctypes.data,
                                 ou.ctypes.data, stt.ctypes.data, _stream(stream)))
    return dict(x=x, J=J, C=C, lam=lam, evals=ev, outer=ou, status=stt)
