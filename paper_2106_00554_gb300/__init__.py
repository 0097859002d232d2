"""GB300-native fast products with the Walsh -> boundary-wavelet change of basis.

Paper: V. Antun, "Recovering wavelet coefficients from binary samples using
fast transforms", arXiv 2106.00554.  The computation lives in libuw.so (CUDA
for sm_103a behind the C ABI of include/uw.h); this package only marshals
arguments.  PyTorch supplies device memory and streams.

    plan = Plan(d=2, R=11, q=1, p=8, boundary=VMP, omega=omega)
    y = plan.forward(x)        # y = P_Omega U x
    z = plan.adjoint(y)        # z = U^* P_Omega^* y
"""
from . import _lib
from ._lib import (UW_BOUNDARY_PERIODIC, UW_BOUNDARY_VMP, UW_F32, UW_F32_SPLIT_BF16, UW_F64,
                   UWError, uw_adjoint, uw_adjoint_host, uw_forward, uw_forward_host, uw_forward_noalloc,
                   uw_host_table,
                   uw_plan_create, uw_plan_destroy, uw_plan_reserve, uw_plan_set_coarsest,
                   uw_plan_set_mask, uw_plan_table)

PERIODIC, VMP = UW_BOUNDARY_PERIODIC, UW_BOUNDARY_VMP
F64, F32, F32_SPLIT_BF16 = UW_F64, UW_F32, UW_F32_SPLIT_BF16


def _stream_ptr(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


class Plan:
    """Owns one uw_plan (tables, mask and workspace on the current device)."""

    def __init__(self, d, R, q, p, boundary=VMP, J0=None, omega=None, max_batch=1, symlet=False):
        """symlet: the least-asymmetric Daubechies filter with p vanishing
        moments (UW_FILTER_SYMLET) instead of the extremal-phase one."""
        self.d, self.R, self.q, self.p, self.boundary, self.symlet = d, R, q, p, boundary, symlet
        self._h = uw_plan_create(d, R, q, p | (_lib.UW_FILTER_SYMLET if symlet else 0), boundary)
        if J0 is not None:
            uw_plan_set_coarsest(self._h, J0)
        if omega is not None:
            uw_plan_set_mask(self._h, omega)
        if max_batch > 1:
            uw_plan_reserve(self._h, max_batch)
        self.max_batch = max_batch

    # -- properties -----------------------------------------------------------
    @property
    def M(self):
        return 1 << self.R

    @property
    def N(self):
        return 1 << (self.R + self.q)

    @property
    def J0(self):
        return _lib.lib().uw_plan_coarsest(self._h)

    @property
    def m(self):
        return _lib.lib().uw_plan_num_samples(self._h)

    @property
    def coeffs(self):
        return _lib.lib().uw_plan_num_coeffs(self._h)

    @property
    def last_launches(self):
        return _lib.lib().uw_plan_last_launches(self._h)

    def set_mask(self, omega):
        uw_plan_set_mask(self._h, omega)

    def reserve(self, max_batch):
        uw_plan_reserve(self._h, max_batch)
        self.max_batch = max_batch

    def table(self, which):
        return uw_plan_table(self._h, which)

    # -- products on device tensors ---------------------------------------------
    @staticmethod
    def _prec(t, precision):
        import torch
        if precision is None:
            return F64 if t.dtype == torch.float64 else F32
        return precision

    def forward(self, x, y=None, precision=None, stream=None):
        """y = P_Omega U x for x of shape (batch, M) / (batch, M, M) or without
        the batch axis; float64 -> UW_F64, float32 -> UW_F32 unless given."""
        import torch
        prec = self._prec(x, precision)
        batch = x.numel() // self.coeffs
        assert x.is_cuda and x.is_contiguous() and batch * self.coeffs == x.numel()
        shape = (batch, self.m) if x.dim() > self.d else (self.m,)
        if y is None:
            y = torch.empty(shape, dtype=x.dtype, device=x.device)
        uw_forward(self._h, prec, x.data_ptr(), y.data_ptr(), batch, _stream_ptr(stream))
        return y

    def forward_noalloc(self, x, y, precision=None, stream=None):
        """uw_forward_noalloc: the 2D forward product into the caller's y with
        the library's fixed scratch (no device allocation in the call)."""
        prec = self._prec(x, precision)
        batch = x.numel() // self.coeffs
        assert x.is_cuda and x.is_contiguous() and batch * self.coeffs == x.numel()
        assert y.is_cuda and y.is_contiguous() and y.numel() == batch * self.m and y.dtype == x.dtype
        uw_forward_noalloc(self._h, prec, x.data_ptr(), y.data_ptr(), batch, _stream_ptr(stream))
        return y

    def adjoint(self, y, x=None, precision=None, stream=None):
        """x = U^* P_Omega^* y for y of shape (batch, m) or (m,)."""
        import torch
        prec = self._prec(y, precision)
        batch = (y.numel() // self.m) if self.m > 0 else (y.shape[0] if y.dim() > 1 else 1)
        assert y.is_cuda and y.is_contiguous() and batch * self.m == y.numel()
        shp = (self.M,) * self.d
        shape = (batch, *shp) if y.dim() > 1 else shp
        if x is None:
            x = torch.empty(shape, dtype=y.dtype, device=y.device)
        uw_adjoint(self._h, prec, y.data_ptr(), x.data_ptr(), batch, _stream_ptr(stream))
        return x

    # -- products on host arrays (copies inside the call) -------------------------
    def forward_host(self, x, y, precision, batch, stream=None):
        uw_forward_host(self._h, precision, x, y, batch, _stream_ptr(stream))

    def adjoint_host(self, y, x, precision, batch, stream=None):
        uw_adjoint_host(self._h, precision, y, x, batch, _stream_ptr(stream))

    def forward_host_async(self, x, y, precision, batch, stream=None):
        _lib.uw_forward_host_async(self._h, precision, x, y, batch, _stream_ptr(stream))

    def adjoint_host_async(self, y, x, precision, batch, stream=None):
        _lib.uw_adjoint_host_async(self._h, precision, y, x, batch, _stream_ptr(stream))

    def host_wait(self):
        _lib.uw_host_wait(self._h)

    def close(self):
        if getattr(self, "_h", None):
            uw_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PlanGroup:
    """uw_group over existing Plans (uneven sizes allowed): one call issues
    every instance's product, spread over `nstreams` internal streams forked
    from and joined back into the caller's stream (capturable as one graph).
    While the group exists its plans run their coarse 2D levels one launch
    per level.  tune() keeps, per plan, the faster line-operator variant."""

    def __init__(self, plans, nstreams=8):
        self.plans = list(plans)
        self._g = _lib.uw_group_create([pl._h for pl in self.plans], nstreams)

    def forward(self, xs, ys, precision, stream=None):
        _lib.uw_group_forward(self._g, precision, [x.data_ptr() for x in xs], [y.data_ptr() for y in ys],
                              _stream_ptr(stream))

    def adjoint(self, ys, xs, precision, stream=None):
        _lib.uw_group_adjoint(self._g, precision, [y.data_ptr() for y in ys], [x.data_ptr() for x in xs],
                              _stream_ptr(stream))

    def tune(self, xs, ys, precision, reps=3, stream=None, cache=None):
        """Overwrites xs and ys (each pair maps x -> y -> x).  For FP32 groups
        on the persistent launch, also picks its parameters and the faster of
        the persistent launch and the forked streams; `cache`: JSON file of
        choices (read first, written after a miss)."""
        _lib.uw_group_tune_cached(self._g, precision, [x.data_ptr() for x in xs], [y.data_ptr() for y in ys], reps,
                                  cache, _stream_ptr(stream))

    def params(self):
        """{'persistent_available', 'persistent_in_use', 'lines_per_task',
        'cols_per_task', 'tiles_per_task', 'radix', 'ctas_per_sm'}"""
        v = _lib.uw_group_params(self._g)
        keys = ("persistent_available", "persistent_in_use", "lines_per_task", "cols_per_task", "tiles_per_task",
                "radix", "ctas_per_sm")
        return dict(zip(keys, v))

    def device_status(self):
        """UW_OK, or UW_ERR_TIMEOUT if a bounded wait of the persistent launch
        gave up since the last query (synchronises the device)."""
        return _lib.uw_group_device_status(self._g)

    def close(self):
        if self._g:
            _lib.uw_group_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
