"""Python front end of libse: a plan object over the C ABI of include/se.h.

PyTorch supplies device memory and streams; every step of the computation
runs in libse's CUDA kernels (and cuFFT).  Each call is issued on torch's
current CUDA stream, so it is ordered with surrounding torch work.
"""
import ctypes

import numpy as np
import torch

from . import _native as nat

PRECISIONS = {"fp64": nat.SE_FP64, "fp32": nat.SE_FP32, "fp32plain": nat.SE_FP32_PLAIN}
FORCE_MODES = {"analytic": nat.SE_FORCE_ANALYTIC, "ik": nat.SE_FORCE_IK}
_TORCH_DTYPE = {nat.SE_FP64: torch.float64, nat.SE_FP32: torch.float32,
                nat.SE_FP32_PLAIN: torch.float32}
_NP_DTYPE = {nat.SE_FP64: np.float64, nat.SE_FP32: np.float32, nat.SE_FP32_PLAIN: np.float32}


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Plan:
    """SE k-space plan for N particles in [0, L)^3 (xi, grid M^3, support P).

    precision: "fp64" (every step in double) or "fp32" (single precision with
    compensated grid sums; FP64 Green's function table and energy reduction).
    force_mode: "analytic" (derivative of the window, Sec. 3.1) or "ik"
    (differentiation in Fourier space, Sec. 2.3; see se_plan_set_force_mode).
    """

    def __init__(self, N, L, xi, M, P, precision="fp64", c=None, eta=None,
                 prefactor=None, spread_variant=0, tile=0, force_mode="analytic"):
        if not torch.cuda.is_available():
            raise RuntimeError("libse needs a CUDA device; none is available")
        self._lib = nat.load()
        self._h = ctypes.c_void_p()
        nat.check(self._lib.se_plan_create(ctypes.byref(self._h), int(N), float(L),
                                           float(xi), int(M), int(P)), "se_plan_create")
        self.N, self.L, self.xi, self.M, self.P = int(N), float(L), float(xi), int(M), int(P)
        self.prec = PRECISIONS[precision]
        nat.check(self._lib.se_plan_set_precision(self._h, self.prec), "se_plan_set_precision")
        if c is not None:
            nat.check(self._lib.se_plan_set_shape(self._h, float(c), 0), "se_plan_set_shape")
        if eta is not None:
            nat.check(self._lib.se_plan_set_shape(self._h, float(eta), 1), "se_plan_set_shape")
        if prefactor is not None:
            nat.check(self._lib.se_plan_set_prefactor(self._h, float(prefactor)),
                      "se_plan_set_prefactor")
        if spread_variant or tile:
            nat.check(self._lib.se_plan_set_tuning(self._h, int(spread_variant), int(tile)),
                      "se_plan_set_tuning")
        self.force_mode = nat.SE_FORCE_ANALYTIC
        if force_mode != "analytic":
            self.set_force_mode(force_mode)
        self.last_status = 0
        self._stream_handle = None   # the stream last handed to the library
        # counts evaluations that overwrite the plan's grids (spreads); the
        # autograd layer uses it to know whether the grid of a forward pass
        # is still in place at its backward pass
        self.generation = 0

    # -- bookkeeping -------------------------------------------------------
    @property
    def dtype(self):
        return _TORCH_DTYPE[self.prec]

    @property
    def np_dtype(self):
        return _NP_DTYPE[self.prec]

    def params(self):
        out = (ctypes.c_double * 10)()
        nat.check(self._lib.se_plan_get_params(self._h, out), "se_plan_get_params")
        keys = ["h", "w", "eta", "alpha", "cg", "m", "tile", "spread_variant", "precision",
                "prefactor"]
        return dict(zip(keys, list(out)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.se_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        # hand torch's current stream to the library when it changed (the
        # library keeps it; a call per step would cost a host round trip)
        s = torch.cuda.current_stream().cuda_stream
        if s != self._stream_handle:
            nat.check(self._lib.se_plan_set_stream(self._h, ctypes.c_void_p(s)),
                      "se_plan_set_stream")
            self._stream_handle = s

    def _check_inputs(self, xyz, q):
        if xyz.dtype != self.dtype or q.dtype != self.dtype:
            raise TypeError("xyz and q must be %s" % self.dtype)
        if not (xyz.is_cuda and q.is_cuda):
            raise TypeError("xyz and q must be CUDA tensors")
        if tuple(xyz.shape) != (self.N, 3) or tuple(q.shape) != (self.N,):
            raise ValueError("expected xyz [%d, 3] and q [%d]" % (self.N, self.N))
        if not (xyz.is_contiguous() and q.is_contiguous()):
            raise ValueError("xyz and q must be contiguous")

    # -- the five steps ----------------------------------------------------
    def spread(self, xyz, q):
        self._check_inputs(xyz, q)
        self._stream()
        self.generation += 1
        nat.check(self._lib.se_spread(self._h, _ptr(xyz), _ptr(q)), "se_spread")

    def scale(self, E_grid=None):
        """FFT, Green's-function scaling, inverse FFT.  E_grid: optional CUDA
        float64 tensor of one element receiving the grid energy."""
        self._stream()
        nat.check(self._lib.se_scale(self._h, _ptr(E_grid)), "se_scale")

    def gather(self, xyz, q, phi=None, F=None, E=None):
        self._check_inputs(xyz, q)
        self._stream()
        nat.check(self._lib.se_gather(self._h, _ptr(xyz), _ptr(q), _ptr(phi), _ptr(F), _ptr(E)),
                  "se_gather")

    def energy_force(self, xyz, q, with_phi=True, F=None, phi=None):
        """E (python float), F [N,3], phi [N] (CUDA tensors of the plan's dtype)."""
        self._check_inputs(xyz, q)
        if F is None:
            F = torch.empty((self.N, 3), dtype=self.dtype, device=xyz.device)
        if phi is None and with_phi:
            phi = torch.empty((self.N,), dtype=self.dtype, device=xyz.device)
        self._stream()
        self.generation += 1
        E = ctypes.c_double()
        st = self._lib.se_energy_force(self._h, _ptr(xyz), _ptr(q), ctypes.byref(E), _ptr(F),
                                       _ptr(phi))
        self.last_status = nat.check(st, "se_energy_force")
        return E.value, F, phi

    def energy(self, xyz, q):
        """Energy-only mode: E (python float) from the grid energy, no gather."""
        self._check_inputs(xyz, q)
        self._stream()
        self.generation += 1
        E = ctypes.c_double()
        st = self._lib.se_energy_force(self._h, _ptr(xyz), _ptr(q), ctypes.byref(E), None, None)
        self.last_status = nat.check(st, "se_energy_force")
        return E.value

    def potential(self, xyz, q, phi=None):
        """Potential-only mode: E (python float) and phi [N] with the plain window
        (no force sums)."""
        self._check_inputs(xyz, q)
        if phi is None:
            phi = torch.empty((self.N,), dtype=self.dtype, device=xyz.device)
        self._stream()
        self.generation += 1
        E = ctypes.c_double()
        st = self._lib.se_energy_force(self._h, _ptr(xyz), _ptr(q), ctypes.byref(E), None,
                                       _ptr(phi))
        self.last_status = nat.check(st, "se_energy_force")
        return E.value, phi

    def energy_force_host(self, xyz, q):
        """Host (numpy) in, host out: copies to the device, evaluates, copies back."""
        xyz = np.ascontiguousarray(xyz, dtype=self.np_dtype)
        q = np.ascontiguousarray(q, dtype=self.np_dtype)
        F = np.empty((self.N, 3), dtype=self.np_dtype)
        phi = np.empty((self.N,), dtype=self.np_dtype)
        self._stream()
        self.generation += 1
        E = ctypes.c_double()
        st = self._lib.se_energy_force_host(
            self._h, xyz.ctypes.data_as(ctypes.c_void_p), q.ctypes.data_as(ctypes.c_void_p),
            ctypes.byref(E), F.ctypes.data_as(ctypes.c_void_p),
            phi.ctypes.data_as(ctypes.c_void_p))
        self.last_status = nat.check(st, "se_energy_force_host")
        return E.value, F, phi

    def energy_force_host_ptrs(self, xyz_ptr, q_ptr, F_ptr, phi_ptr):
        """se_energy_force_host on raw host pointers (e.g. pinned torch tensors)."""
        self._stream()
        self.generation += 1
        E = ctypes.c_double()
        st = self._lib.se_energy_force_host(self._h, ctypes.c_void_p(xyz_ptr),
                                            ctypes.c_void_p(q_ptr), ctypes.byref(E),
                                            ctypes.c_void_p(F_ptr), ctypes.c_void_p(phi_ptr))
        self.last_status = nat.check(st, "se_energy_force_host")
        return E.value

    STAGES = ("bin", "scatter", "spread", "fft_fwd", "scale", "fft_inv", "gather")

    def set_timing(self, enable=True):
        nat.check(self._lib.se_plan_set_timing(self._h, int(bool(enable))), "se_plan_set_timing")

    def get_timing(self, reset=True):
        """(summed ms per stage as a dict, number of evaluations summed)."""
        ms = (ctypes.c_double * 7)()
        n = ctypes.c_int64()
        nat.check(self._lib.se_plan_get_timing(self._h, ms, 7, ctypes.byref(n), int(reset)),
                  "se_plan_get_timing")
        return dict(zip(self.STAGES, list(ms))), n.value

    def evaluate(self, xyz, q, F=None, phi=None, E=None):
        """se_evaluate: the whole evaluation with results on the device and no
        host synchronisation (E: optional CUDA float64 tensor of one element).
        Arguments are not re-checked here (hot path)."""
        self._stream()
        self.generation += 1
        nat.check(self._lib.se_evaluate(self._h, _ptr(xyz), _ptr(q), _ptr(F), _ptr(phi), _ptr(E)),
                  "se_evaluate")

    def adjoint(self, xyz, q, gE, grad_x=None, grad_q=None):
        """se_adjoint: grad_x = -g F, grad_q = g phi for g = gE (CUDA float64, one
        element), from the grid of the last scale() of this plan."""
        self._stream()
        nat.check(self._lib.se_adjoint(self._h, _ptr(xyz), _ptr(q), _ptr(gE), _ptr(grad_x),
                                       _ptr(grad_q)), "se_adjoint")

    def status(self):
        st = ctypes.c_int()
        nat.check(self._lib.se_plan_get_status(self._h, ctypes.byref(st)), "se_plan_get_status")
        return st.value

    def set_graph(self, enable=True):
        nat.check(self._lib.se_plan_set_graph(self._h, int(bool(enable))), "se_plan_set_graph")

    def set_tile(self, tile):
        """Spreading tile edge (grid cells); keeps the automatic pipeline choice."""
        nat.check(self._lib.se_plan_set_tuning(self._h, 0, int(tile)), "se_plan_set_tuning")

    def set_tuning(self, spread_variant, tile=0):
        """Spreading variant (0 automatic, 1-4 as in se_plan_set_tuning) and tile edge."""
        nat.check(self._lib.se_plan_set_tuning(self._h, int(spread_variant), int(tile)),
                  "se_plan_set_tuning")

    def set_force_mode(self, mode):
        """"analytic" or "ik" (or SE_FORCE_ANALYTIC / SE_FORCE_IK)."""
        m = FORCE_MODES[mode] if isinstance(mode, str) else int(mode)
        nat.check(self._lib.se_plan_set_force_mode(self._h, m), "se_plan_set_force_mode")
        self.force_mode = m

    def copy_grid(self, which):
        """0: spread grid H (valid after spread), 1: Ht (after scale); [M,M,M] tensor."""
        out = torch.empty((self.M, self.M, self.M), dtype=self.dtype, device="cuda")
        self._stream()
        nat.check(self._lib.se_copy_grid(self._h, int(which), _ptr(out)), "se_copy_grid")
        return out

    def self_energy(self, q):
        q = np.ascontiguousarray(np.asarray(q, dtype=np.float64))
        E = ctypes.c_double()
        nat.check(self._lib.se_self_energy(self._h, q.ctypes.data_as(ctypes.c_void_p), len(q),
                                           ctypes.byref(E)), "se_self_energy")
        return E.value


class RealSpace:
    """Real-space part of the Ewald sum with cell lists (se_real_*): phi, F and
    E of the erfc terms within rc plus the self term, on the GPU; added to a
    Plan's k-space results they give the whole Ewald sum."""

    def __init__(self, N, L, xi, rc, precision="fp64", prefactor=None):
        if not torch.cuda.is_available():
            raise RuntimeError("libse needs a CUDA device; none is available")
        self._lib = nat.load()
        self._h = ctypes.c_void_p()
        nat.check(self._lib.se_real_create(ctypes.byref(self._h), int(N), float(L), float(xi),
                                           float(rc)), "se_real_create")
        self.N = int(N)
        self.prec = PRECISIONS[precision]
        if self.prec == nat.SE_FP32_PLAIN:
            self.prec = nat.SE_FP32
        nat.check(self._lib.se_real_set_precision(self._h, self.prec), "se_real_set_precision")
        if prefactor is not None:
            nat.check(self._lib.se_real_set_prefactor(self._h, float(prefactor)),
                      "se_real_set_prefactor")

    @property
    def dtype(self):
        return _TORCH_DTYPE[self.prec]

    def set_reach(self, K):
        """Stencil reach 1-3 (cells of edge >= rc/K), 0 automatic."""
        nat.check(self._lib.se_real_set_reach(self._h, int(K)), "se_real_set_reach")

    def cells_per_dim(self):
        n = ctypes.c_int()
        nat.check(self._lib.se_real_get_cells(self._h, ctypes.byref(n)), "se_real_get_cells")
        return n.value

    def evaluate(self, xyz, q, F=None, phi=None, E=None, accumulate=False):
        """Device tensors (plan dtype); E: CUDA float64 tensor of one element."""
        if self.N > 0:
            for name, t, shape in (("xyz", xyz, (self.N, 3)), ("q", q, (self.N,)),
                                   ("F", F, (self.N, 3)), ("phi", phi, (self.N,))):
                if t is None:
                    if name in ("xyz", "q"):
                        raise ValueError("%s is required" % name)
                    continue
                if t.dtype != self.dtype or not t.is_cuda or not t.is_contiguous() or \
                        tuple(t.shape) != shape:
                    raise TypeError("%s must be a contiguous CUDA %s tensor of shape %s"
                                    % (name, self.dtype, shape))
        if E is not None and (E.dtype != torch.float64 or not E.is_cuda or E.numel() < 1):
            raise TypeError("E must be a CUDA float64 tensor")
        s = torch.cuda.current_stream().cuda_stream
        nat.check(self._lib.se_real_set_stream(self._h, ctypes.c_void_p(s)), "se_real_set_stream")
        nat.check(self._lib.se_real_evaluate(self._h, _ptr(xyz), _ptr(q), _ptr(F), _ptr(phi),
                                             _ptr(E), int(bool(accumulate))), "se_real_evaluate")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.se_real_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


QUANTITIES = {"potential": nat.SE_QUANTITY_POTENTIAL, "energy": nat.SE_QUANTITY_ENERGY,
              "force": nat.SE_QUANTITY_FORCE}


def select_params(quantity, tol, rc, L, Q, c=0.95):
    """se_select_params (host only, no device needed): xi, M, P for an absolute
    rms error tol of "potential", "energy" or "force" with real-space cut-off
    rc, box L and Q = sum q^2.  Returns dict(xi, M, P, k_inf, supported);
    supported is False when P would exceed 32 or no Fourier part is needed."""
    lib = nat.load()
    xi, kinf = ctypes.c_double(), ctypes.c_double()
    M, P = ctypes.c_int(), ctypes.c_int()
    qn = QUANTITIES[quantity] if isinstance(quantity, str) else int(quantity)
    st = lib.se_select_params(qn, float(tol), float(rc), float(L), float(Q), float(c),
                              ctypes.byref(xi), ctypes.byref(M), ctypes.byref(P),
                              ctypes.byref(kinf))
    if st == nat.SE_ERR_UNSUPPORTED:
        return dict(xi=xi.value, M=M.value, P=P.value, k_inf=kinf.value, supported=False)
    nat.check(st, "se_select_params")
    return dict(xi=xi.value, M=M.value, P=P.value, k_inf=kinf.value, supported=True)


def select_support(scaled_tol, c=0.95):
    """se_select_support: smallest even P with e^{-pi P c^2/2} <= scaled_tol."""
    return nat.check(nat.load().se_select_support(float(scaled_tol), float(c)),
                     "se_select_support")


def lambert_w0(z):
    return nat.load().se_lambert_w0(float(z))


# C-ABI names, for callers who want the flat interface.
def se_plan_create(N, L, xi, M, P, **kw):
    return Plan(N, L, xi, M, P, **kw)


def se_spread(plan, xyz, q):
    return plan.spread(xyz, q)


def se_scale(plan, E_grid=None):
    return plan.scale(E_grid)


def se_gather(plan, xyz, q, phi=None, F=None, E=None):
    return plan.gather(xyz, q, phi, F, E)


def se_energy_force(plan, xyz, q, **kw):
    return plan.energy_force(xyz, q, **kw)


def se_energy_force_host(plan, xyz, q):
    return plan.energy_force_host(xyz, q)


def se_plan_destroy(plan):
    plan.close()


class Batch:
    """S independent systems evaluated together (se_batch_*): Ns, Ls, Ms per
    system, common xi and P; float32 arrays concatenated over the systems."""

    def __init__(self, Ns, Ls, Ms, xi, P, tile=None, prefactor=None):
        if not torch.cuda.is_available():
            raise RuntimeError("libse needs a CUDA device; none is available")
        self._lib = nat.load()
        self.S = len(Ns)
        self.Ns = np.asarray(Ns, dtype=np.int64)
        self.Ls = np.asarray(Ls, dtype=np.float64)
        self.Ms = np.asarray(Ms, dtype=np.int32)
        self.xi, self.P = float(xi), int(P)
        self.offsets = np.concatenate([[0], np.cumsum(self.Ns)])
        self.Ntot = int(self.offsets[-1])
        self._h = ctypes.c_void_p()
        nat.check(self._lib.se_batch_create(
            ctypes.byref(self._h), self.S, self.Ns.ctypes.data_as(ctypes.c_void_p),
            self.Ls.ctypes.data_as(ctypes.c_void_p), self.Ms.ctypes.data_as(ctypes.c_void_p),
            self.xi, self.P), "se_batch_create")
        if tile:
            nat.check(self._lib.se_batch_set_tile(self._h, int(tile)), "se_batch_set_tile")
        if prefactor is not None:
            nat.check(self._lib.se_batch_set_prefactor(self._h, float(prefactor)),
                      "se_batch_set_prefactor")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.se_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        s = torch.cuda.current_stream().cuda_stream
        nat.check(self._lib.se_batch_set_stream(self._h, ctypes.c_void_p(s)), "se_batch_set_stream")

    def set_graph(self, enable=True):
        nat.check(self._lib.se_batch_set_graph(self._h, int(bool(enable))), "se_batch_set_graph")

    def set_tile(self, tile):
        nat.check(self._lib.se_batch_set_tile(self._h, int(tile)), "se_batch_set_tile")

    def evaluate(self, xyz, q, F=None, phi=None, E=None):
        """Returns (E [S] float64, F [Ntot,3], phi [Ntot]) CUDA tensors."""
        if F is None:
            F = torch.empty((self.Ntot, 3), dtype=torch.float32, device=xyz.device)
        if phi is None:
            phi = torch.empty((self.Ntot,), dtype=torch.float32, device=xyz.device)
        if E is None:
            E = torch.empty((self.S,), dtype=torch.float64, device=xyz.device)
        self._stream()
        nat.check(self._lib.se_batch_evaluate(self._h, _ptr(xyz), _ptr(q), _ptr(F), _ptr(phi),
                                              _ptr(E)), "se_batch_evaluate")
        return E, F, phi

    def grid_energy(self):
        Eg = torch.empty((self.S,), dtype=torch.float64, device="cuda")
        self._stream()
        nat.check(self._lib.se_batch_grid_energy(self._h, _ptr(Eg)), "se_batch_grid_energy")
        return Eg

    STAGES = ("bin", "scatter", "spread", "fft_fwd", "scale", "fft_inv", "gather", "finish")

    def set_timing(self, enable=True):
        nat.check(self._lib.se_batch_set_timing(self._h, int(bool(enable))), "se_batch_set_timing")

    def get_timing(self, reset=True):
        """(summed ms per stage as a dict, number of evaluations timed)."""
        ms = (ctypes.c_double * 8)()
        n = ctypes.c_int64()
        nat.check(self._lib.se_batch_get_timing(self._h, ms, 8, ctypes.byref(n), int(reset)),
                  "se_batch_get_timing")
        return dict(zip(self.STAGES, list(ms))), n.value

    def status(self):
        st = ctypes.c_int()
        nat.check(self._lib.se_batch_get_status(self._h, ctypes.byref(st)), "se_batch_get_status")
        return st.value

    def autotune(self, xyz, q, candidates=(4, 6, 8, 10), reps=10):
        """Time each tile edge and keep the fastest; returns (tile, ms per evaluation)."""
        c = np.asarray(candidates, dtype=np.int32)
        F = torch.empty((self.Ntot, 3), dtype=torch.float32, device=xyz.device)
        phi = torch.empty((self.Ntot,), dtype=torch.float32, device=xyz.device)
        E = torch.empty((self.S,), dtype=torch.float64, device=xyz.device)
        best = ctypes.c_int()
        ms = ctypes.c_float()
        self._stream()
        nat.check(self._lib.se_batch_autotune(self._h, _ptr(xyz), _ptr(q), _ptr(F), _ptr(phi),
                                              _ptr(E), c.ctypes.data_as(ctypes.c_void_p), len(c),
                                              int(reps), ctypes.byref(best), ctypes.byref(ms)),
                  "se_batch_autotune")
        return best.value, ms.value


def probe_peak(kind):
    """se_probe_peak: measured rate of one GPU unit on the current device
    (kind: "fp32_fma" or "fp64_fma" in flop/s, "smem_atomic_u32" or
    "smem_atomic_f32" in shared-memory atomic adds per second)."""
    kinds = {"fp32_fma": nat.SE_PROBE_FP32_FMA, "fp64_fma": nat.SE_PROBE_FP64_FMA,
             "smem_atomic_u32": nat.SE_PROBE_SMEM_ATOMIC_U32,
             "smem_atomic_f32": nat.SE_PROBE_SMEM_ATOMIC_F32}
    out = ctypes.c_double()
    nat.check(nat.load().se_probe_peak(kinds[kind], ctypes.byref(out)), "se_probe_peak")
    return out.value
