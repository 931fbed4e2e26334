"""Argument marshalling for the C ABI (no arithmetic of the method here)."""
from __future__ import annotations

import ctypes

import torch

from . import _native as nat

PREC_FP64 = 0
PREC_MIXED = 1
PREC_MIXED_FULL = 2
_PREC = {"fp64": PREC_FP64, "mixed": PREC_MIXED, "mixed_full": PREC_MIXED_FULL, PREC_FP64: PREC_FP64,
         PREC_MIXED: PREC_MIXED, PREC_MIXED_FULL: PREC_MIXED_FULL}


class TTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ttround error {code}: {msg}")
        self.code = code


def _check(rc):
    if rc != 0:
        raise TTError(rc, nat.last_error())


def _i64(vals):
    vals = [int(v) for v in vals]
    return (ctypes.c_int64 * max(len(vals), 1))(*vals)


def _ptrs(tensors):
    return (ctypes.c_void_p * max(len(tensors), 1))(*[t.data_ptr() for t in tensors])


def _stream(stream, device):
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return ctypes.c_void_p(s.cuda_stream)


def _check_core(t, name, dtype=torch.float64):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.dim() == 3
            and t.is_contiguous()):
        raise ValueError(f"{name}: expected a contiguous {dtype} CUDA tensor of shape (r0, I, r1)")


def tt_version() -> str:
    return nat.lib().tt_version().decode()


def tt_sketch_gaussian(dims, ells, seed, *, device=None, stream=None):
    """Gaussian TT of Definition 3.1 drawn on the device (Philox4x32-10)."""
    dims = [int(d) for d in dims]
    N = len(dims)
    device = torch.device(device or "cuda")
    out = [torch.empty((int(ells[n]), dims[n], int(ells[n + 1])), dtype=torch.float64, device=device)
           for n in range(N)]
    _check(nat.lib().tt_sketch_gaussian(N, _i64(dims), _i64(ells), ctypes.c_uint64(int(seed)), _ptrs(out),
                                        _stream(stream, device)))
    return out


def tt_gemm_emulated_f64(A, B, C=None, *, alpha=1.0, beta=0.0, digits=8, stream=None):
    """C = alpha A B + beta C by the emulated FP64 tensor-core product (2-D float64
    CUDA tensors with any strides; C is created when None)."""
    for t, nm in ((A, "A"), (B, "B")):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.dim() == 2):
            raise ValueError(f"{nm}: expected a 2-D float64 CUDA tensor")
    M, K = A.shape
    K2, N = B.shape
    if K != K2:
        raise ValueError("inner dimensions differ")
    if C is None:
        C = torch.zeros((M, N), dtype=torch.float64, device=A.device)
    elif not (C.is_cuda and C.dtype == torch.float64 and tuple(C.shape) == (M, N)):
        raise ValueError("C: expected a float64 CUDA tensor of shape (M, N)")
    _check(nat.lib().tt_gemm_emulated_f64(M, N, K, float(alpha), A.data_ptr(), A.stride(0), A.stride(1),
                                          B.data_ptr(), B.stride(0), B.stride(1), float(beta), C.data_ptr(),
                                          C.stride(0), C.stride(1), int(digits), None, 0, _stream(stream, A.device)))
    return C


def clamp_ranks(dims, ells):
    N = len(dims)
    ell = [1] + [int(x) for x in ells[1:N]] + [1]
    for n in range(1, N):
        ell[n] = min(ell[n], ell[n - 1] * dims[n - 1])
    for n in range(N - 1, 0, -1):
        ell[n] = min(ell[n], ell[n + 1] * dims[n])
    return ell


def tt_round_sum_rand(summands, ells, *, tol=0.0, sketch=None, seed=0, coeffs=None, precision="fp64",
                      workspace=None, stream=None):
    """Algorithm 7 (sum of TTs, Randomize-then-Orthogonalize) on the GPU.

    summands: list of K TTs (lists of N cores). ells: N+1 target ranks.
    sketch: optional list of N sketch cores (l_{n-1}, I_n, l_n); None draws it
    on the device from seed. Returns the list of output cores."""
    K = len(summands)
    N = len(summands[0])
    device = summands[0][0].device
    dims = [int(c.shape[1]) for c in summands[0]]
    ranks = []
    flat = []
    for j, Y in enumerate(summands):
        if len(Y) != N:
            raise ValueError("all summands need the same order")
        ranks += [int(Y[0].shape[0])] + [int(c.shape[2]) for c in Y]
        for n, c in enumerate(Y):
            _check_core(c, f"summand {j} core {n}")
            if int(c.shape[1]) != dims[n]:
                raise ValueError("mode sizes differ between summands")
    for Y in summands:
        flat += list(Y)
    ell = clamp_ranks(dims, ells)
    out = [torch.empty((ell[n], dims[n], ell[n + 1]), dtype=torch.float64, device=device) for n in range(N)]
    sk_arr = None
    if sketch is not None:
        for n, c in enumerate(sketch):
            _check_core(c, f"sketch core {n}")
            if tuple(c.shape) != (ell[n], dims[n], ell[n + 1]):
                raise ValueError(f"sketch core {n} has shape {tuple(c.shape)}, expected "
                                 f"{(ell[n], dims[n], ell[n + 1])}")
        sk_arr = _ptrs(sketch)
    co = None
    if coeffs is not None:
        co = (ctypes.c_double * K)(*[float(c) for c in coeffs])
    prec = _PREC[precision]
    L = nat.lib()
    dims_a, ranks_a, ell_a = _i64(dims), _i64(ranks), _i64(ell)
    ws_bytes = 0
    ws_ptr = None
    if workspace is None:
        ws_bytes = L.tt_round_sum_rand_workspace(N, K, dims_a, ranks_a, ell_a, float(tol), prec)
        if ws_bytes == 0:
            _check(L.tt_round_sum_rand(N, K, dims_a, ranks_a, _ptrs(flat), co, ell_a, sk_arr, 0, float(tol), prec,
                                       None, None, None, 0, None) or 1)
        workspace = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=device)
    ws_ptr = workspace.data_ptr()
    ws_ptr += (-ws_ptr) % 256
    ws_bytes = workspace.numel() - (ws_ptr - workspace.data_ptr())
    out_ranks = (ctypes.c_int64 * (N + 1))()
    _check(L.tt_round_sum_rand(N, K, dims_a, ranks_a, _ptrs(flat), co, ell_a, sk_arr, ctypes.c_uint64(int(seed)),
                               float(tol), prec, _ptrs(out), out_ranks, ctypes.c_void_p(ws_ptr), ws_bytes,
                               _stream(stream, device)))
    r = [int(x) for x in out_ranks]
    res = []
    for n in range(N):
        cnt = r[n] * dims[n] * r[n + 1]
        res.append(out[n].view(-1)[:cnt].view(r[n], dims[n], r[n + 1]))
    return res


_ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class _DeviceView:
    """A float64 device buffer handed to Python through __cuda_array_interface__."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 2, "strides": None}


def tt_round_sum_rand_sharded(summands, ells, allreduce, *, tol=0.0, sketch=None, seed=0, coeffs=None,
                              precision="fp64", workspace=None, stream=None):
    """Algorithm 7 with this rank's share of the summands (tt_round_sum_rand_sharded):
    allreduce(tensor, stream) must replace the float64 CUDA tensor by its sum
    over the ranks, ordered on `stream` (a torch.cuda.ExternalStream), e.g.
    torch.distributed.all_reduce under that stream. Returns the whole rounded
    tensor (the same on every rank)."""
    K = len(summands)
    N = len(summands[0])
    device = summands[0][0].device
    N2, K2, dims, ranks, flat = _sum_args(summands)
    ell = clamp_ranks(dims, ells)
    out = [torch.empty((ell[n], dims[n], ell[n + 1]), dtype=torch.float64, device=device) for n in range(N)]
    sk_arr = _ptrs(sketch) if sketch is not None else None
    co = (ctypes.c_double * K)(*[float(c) for c in coeffs]) if coeffs is not None else None
    err = []

    def cb(ptr, count, strm, ctx):
        try:
            t = torch.as_tensor(_DeviceView(ptr, count), device=device)
            allreduce(t, torch.cuda.ExternalStream(int(strm) if strm else 0, device=device))
            return 0
        except Exception as e:          # reported through the library's status
            err.append(e)
            return 1

    fn = _ALLREDUCE_FN(cb)
    L = nat.lib()
    prec = _PREC[precision]
    dims_a, ranks_a, ell_a = _i64(dims), _i64(ranks), _i64(ell)
    nb = L.tt_round_sum_rand_workspace(N, K, dims_a, ranks_a, ell_a, float(tol), prec)
    if nb == 0:
        raise TTError(1, nat.last_error())
    workspace, wp, wb = _workspace(nb, device, workspace)
    out_ranks = (ctypes.c_int64 * (N + 1))()
    rc = L.tt_round_sum_rand_sharded(N, K, dims_a, ranks_a, _ptrs(flat), co, ell_a, sk_arr,
                                     ctypes.c_uint64(int(seed)), float(tol), prec, _ptrs(out), out_ranks, wp, wb,
                                     _stream(stream, device), ctypes.cast(fn, ctypes.c_void_p), None)
    if err:
        raise err[0]
    _check(rc)
    r = [int(x) for x in out_ranks]
    return [out[n].view(-1)[:r[n] * dims[n] * r[n + 1]].view(r[n], dims[n], r[n + 1]) for n in range(N)]


def tt_round_rand_backward(cores, ells, sketch, xbar, *, workspace=None, stream=None):
    """dL/dY for fixed-sketch RandOrth (Algorithm 5, fixed ranks) given
    xbar = dL/dX_hat for its output cores; returns tensors shaped like cores.
    float32 tensors take the float32 entry point (FP32-class products, FP64
    QR steps)."""
    N = len(cores)
    device = cores[0].device
    dt = cores[0].dtype
    f32 = dt == torch.float32
    dims = [int(c.shape[1]) for c in cores]
    ranks = [int(cores[0].shape[0])] + [int(c.shape[2]) for c in cores]
    for n, c in enumerate(cores):
        _check_core(c, f"core {n}", dt)
    ell = clamp_ranks(dims, ells)
    for n in range(N):
        want = (ell[n], dims[n], ell[n + 1])
        _check_core(xbar[n], f"xbar core {n}", dt)
        if tuple(xbar[n].shape) != want:
            raise ValueError(f"xbar core {n} has shape {tuple(xbar[n].shape)}, expected {want}")
        if n > 0:
            _check_core(sketch[n], f"sketch core {n}", dt)
            if tuple(sketch[n].shape) != want:
                raise ValueError(f"sketch core {n} has shape {tuple(sketch[n].shape)}, expected {want}")
    sk = [sketch[n] if n > 0 else xbar[0] for n in range(N)]     # core 1 of the sketch is not used
    ybar = [torch.empty_like(c) for c in cores]
    L = nat.lib()
    dims_a, ranks_a, ell_a = _i64(dims), _i64(ranks), _i64(ell)
    if f32:
        nbytes = L.tt_round_rand_backward_f32_workspace(N, dims_a, ranks_a, ell_a)
        fn = L.tt_round_rand_backward_f32
    else:
        nbytes = L.tt_round_rand_backward_workspace(N, dims_a, ranks_a, ell_a)
        fn = L.tt_round_rand_backward
    if nbytes == 0 and N > 1:
        raise TTError(1, nat.last_error())
    workspace, wp, wb = _workspace(nbytes, device, workspace)
    _check(fn(N, dims_a, ranks_a, _ptrs(cores), ell_a, _ptrs(sk), _ptrs(xbar), _ptrs(ybar), wp, wb,
              _stream(stream, device)))
    return ybar


class _RandOrthFixedSketch(torch.autograd.Function):
    @staticmethod
    def forward(ctx, ell, sketch, *cores):
        prec = "mixed" if cores[0].dtype == torch.float32 else "fp64"
        out = tt_round_rand(list(cores), ell, sketch=sketch, tol=0.0, precision=prec)
        ctx.save_for_backward(*cores)
        ctx.ell = list(ell)
        ctx.sketch = sketch
        return tuple(o.contiguous() for o in out)

    @staticmethod
    def backward(ctx, *gout):
        cores = ctx.saved_tensors
        ell = clamp_ranks([int(c.shape[1]) for c in cores], ctx.ell)
        xb = [g.contiguous() if g is not None else
              torch.zeros((ell[n], cores[n].shape[1], ell[n + 1]), dtype=cores[0].dtype, device=cores[0].device)
              for n, g in enumerate(gout)]
        ybar = tt_round_rand_backward(list(cores), ctx.ell, ctx.sketch, xb)
        return (None, None, *ybar)


def round_rand_fixed_sketch(cores, ells, sketch):
    """Differentiable fixed-sketch RandOrth (Algorithm 5, fixed ranks): forward
    by tt_round_rand, backward by tt_round_rand_backward (float64, or float32
    cores and sketch with FP32-class products and FP64 QR steps)."""
    return list(_RandOrthFixedSketch.apply(list(ells), list(sketch), *cores))


class SumRoundingPlan:
    """Captured plan of tt_round_sum_rand for fixed mode sizes, summand ranks,
    sketch ranks, tolerance and precision; calling it replays the CUDA graph on
    new summand cores, coefficients and seed (results bit-wise equal to
    tt_round_sum_rand with the same seed)."""

    def __init__(self, dims, summand_ranks, ells, *, tol=0.0, precision="fp64", device=None, stream=None):
        self.dims = [int(d) for d in dims]
        self.N = len(self.dims)
        self.summand_ranks = [[int(r) for r in R] for R in summand_ranks]
        self.K = len(self.summand_ranks)
        self.ell = clamp_ranks(self.dims, ells)
        self.tol = float(tol)
        self.device = torch.device(device or "cuda")
        flat = [r for R in self.summand_ranks for r in R]
        h = ctypes.c_void_p()
        _check(nat.lib().tt_sum_plan_create(self.N, self.K, _i64(self.dims), _i64(flat), _i64(self.ell), self.tol,
                                            _PREC[precision], ctypes.byref(h), _stream(stream, self.device)))
        self._h = h

    @property
    def launches(self):
        return int(nat.lib().tt_sum_plan_launches(self._h))

    def __call__(self, summands, *, seed=0, coeffs=None, out=None, stream=None):
        N, K, dims, ranks, flat = _sum_args(summands)
        if (N, K, dims) != (self.N, self.K, self.dims) or ranks != [r for R in self.summand_ranks for r in R]:
            raise ValueError("summands do not match the plan's sizes and ranks")
        ell = self.ell
        if out is None:
            out = [torch.empty((ell[n], dims[n], ell[n + 1]), dtype=torch.float64, device=self.device)
                   for n in range(N)]
        co = None if coeffs is None else (ctypes.c_double * K)(*[float(c) for c in coeffs])
        out_ranks = (ctypes.c_int64 * (N + 1))()
        _check(nat.lib().tt_sum_plan_run(self._h, _ptrs(flat), co, ctypes.c_uint64(int(seed)), _ptrs(out),
                                         out_ranks, _stream(stream, self.device)))
        r = [int(x) for x in out_ranks]
        return [out[n].view(-1)[:r[n] * dims[n] * r[n + 1]].view(r[n], dims[n], r[n + 1]) for n in range(N)]

    def host_layout(self):
        """(in_offsets K*N, out_offsets N, in_total, out_total) of the packed
        host arrays of run_host, in float64 elements."""
        io = (ctypes.c_int64 * (self.K * self.N))()
        oo = (ctypes.c_int64 * self.N)()
        it, ot = ctypes.c_int64(), ctypes.c_int64()
        _check(nat.lib().tt_sum_plan_host_layout(self._h, io, oo, ctypes.byref(it), ctypes.byref(ot)))
        return list(io), list(oo), int(it.value), int(ot.value)

    def pack_host(self, summands, *, pin=True):
        """One packed float64 host array (pinned by default) of the summands'
        cores (K lists of N arrays / CPU tensors of the plan's shapes)."""
        io, _, it, _ = self.host_layout()
        buf = torch.empty(max(it, 1), dtype=torch.float64, pin_memory=pin)
        if len(summands) != self.K:
            raise ValueError("summands do not match the plan's sizes and ranks")
        for j, Y in enumerate(summands):
            for n, c in enumerate(Y):
                t = torch.as_tensor(c, dtype=torch.float64).reshape(-1)
                R = self.summand_ranks[j]
                if t.numel() != R[n] * self.dims[n] * R[n + 1]:
                    raise ValueError("summands do not match the plan's sizes and ranks")
                buf[io[j * self.N + n]:io[j * self.N + n] + t.numel()].copy_(t)
        return buf

    def run_host(self, h_in, *, seed=0, coeffs=None, out=None, stream=None):
        """Replay on host buffers: h_in from pack_host (float64 CPU tensor of
        in_total elements, pinned for full-speed copies), out a float64 CPU
        tensor of out_total elements (allocated pinned if None). One copy in,
        the graph, one copy out; returns the rounded cores as views of out."""
        _, oo, it, ot = self.host_layout()
        if h_in.dtype != torch.float64 or h_in.device.type != "cpu" or not h_in.is_contiguous() or h_in.numel() < it:
            raise ValueError("h_in must be a contiguous float64 CPU tensor of in_total elements")
        if out is None:
            out = torch.empty(max(ot, 1), dtype=torch.float64, pin_memory=True)
        if out.dtype != torch.float64 or out.device.type != "cpu" or not out.is_contiguous() or out.numel() < ot:
            raise ValueError("out must be a contiguous float64 CPU tensor of out_total elements")
        co = None if coeffs is None else (ctypes.c_double * self.K)(*[float(c) for c in coeffs])
        out_ranks = (ctypes.c_int64 * (self.N + 1))()
        _check(nat.lib().tt_sum_plan_run_host(self._h, ctypes.c_void_p(h_in.data_ptr()), co,
                                              ctypes.c_uint64(int(seed)), ctypes.c_void_p(out.data_ptr()), out_ranks,
                                              _stream(stream, self.device)))
        r = [int(x) for x in out_ranks]
        d = self.dims
        return [out[oo[n]:oo[n] + r[n] * d[n] * r[n + 1]].view(r[n], d[n], r[n + 1]) for n in range(self.N)]

    def status(self, stream=None):
        """Waits for the last replay and raises TTError if a kernel reported a
        failure (TT_ETIMEOUT, TT_ESINGULAR)."""
        _check(nat.lib().tt_sum_plan_status(self._h, _stream(stream, self.device)))

    def close(self):
        if getattr(self, "_h", None):
            nat.lib().tt_sum_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _SumProblem(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("K", ctypes.c_int32), ("dims", ctypes.POINTER(ctypes.c_int64)),
                ("ranks", ctypes.POINTER(ctypes.c_int64)), ("ells", ctypes.POINTER(ctypes.c_int64)),
                ("tol", ctypes.c_double)]


class _BatchSchedule(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("qr_ctas", ctypes.c_int32), ("fused", ctypes.c_int32)]


class BatchRoundingPlan:
    """B independent sum roundings captured in one CUDA graph. problems: list
    of dicts with keys dims, summand_ranks (K lists of N+1 ranks), ells (N+1)
    and optionally tol (default 0). Schedule (no effect on the mathematics):
    fused=-1 groups the launches of all problems (fixed ranks) into `width`
    chains with about qr_ctas CTAs per thin QR; fused=0 runs one schedule per
    problem on `width` chains (see tt_batch_plan_create_sched)."""

    def __init__(self, problems, *, precision="mixed", width=1, qr_ctas=8, fused=-1, device=None, stream=None):
        self.device = torch.device(device or "cuda")
        self.problems = []
        keep = []
        arr = (_SumProblem * len(problems))()
        for b, pr in enumerate(problems):
            dims = [int(d) for d in pr["dims"]]
            R = [[int(r) for r in Rj] for Rj in pr["summand_ranks"]]
            ell = clamp_ranks(dims, pr["ells"])
            tol = float(pr.get("tol", 0.0))
            a_d, a_r, a_e = _i64(dims), _i64([r for Rj in R for r in Rj]), _i64(ell)
            keep += [a_d, a_r, a_e]
            arr[b] = _SumProblem(len(dims), len(R), a_d, a_r, a_e, tol)
            self.problems.append(dict(dims=dims, summand_ranks=R, ell=ell, tol=tol))
        self.width = int(width)
        self.qr_ctas = int(qr_ctas)
        sched = _BatchSchedule(self.width, self.qr_ctas, int(fused))
        h = ctypes.c_void_p()
        _check(nat.lib().tt_batch_plan_create_sched(len(problems), ctypes.cast(arr, ctypes.c_void_p),
                                                    _PREC[precision], ctypes.byref(sched), ctypes.byref(h),
                                                    _stream(stream, self.device)))
        self._h = h

    @property
    def fused(self):
        return bool(nat.lib().tt_batch_plan_is_fused(self._h))

    @property
    def launches(self):
        return int(nat.lib().tt_batch_plan_launches(self._h))

    def __call__(self, batch, *, seeds=None, out=None, stream=None):
        """batch: per problem, its list of K summand TTs (device cores)."""
        if len(batch) != len(self.problems):
            raise ValueError("batch size differs from the plan's")
        flat, outs, nrk = [], [], 0
        for b, (summands, pr) in enumerate(zip(batch, self.problems)):
            N, K, dims, ranks, fl = _sum_args(summands)
            if dims != pr["dims"] or ranks != [r for Rj in pr["summand_ranks"] for r in Rj]:
                raise ValueError(f"problem {b} does not match the plan")
            flat += fl
            ell = pr["ell"]
            o = out[b] if out is not None else [
                torch.empty((ell[n], dims[n], ell[n + 1]), dtype=torch.float64, device=self.device) for n in range(N)]
            outs.append(o)
            nrk += N + 1
        sd = None
        if seeds is not None:
            sd = (ctypes.c_uint64 * len(seeds))(*[int(x) for x in seeds])
        rk = (ctypes.c_int64 * nrk)()
        _check(nat.lib().tt_batch_plan_run(self._h, _ptrs(flat), ctypes.cast(sd, ctypes.c_void_p) if sd else None,
                                           _ptrs([c for o in outs for c in o]), rk, _stream(stream, self.device)))
        res, i = [], 0
        for o, pr in zip(outs, self.problems):
            N, dims = len(pr["dims"]), pr["dims"]
            r = [int(rk[i + n]) for n in range(N + 1)]
            i += N + 1
            res.append([o[n].view(-1)[:r[n] * dims[n] * r[n + 1]].view(r[n], dims[n], r[n + 1]) for n in range(N)])
        return res

    def status(self, stream=None):
        """Waits for the last replay and raises TTError if a kernel reported a failure."""
        _check(nat.lib().tt_batch_plan_status(self._h, _stream(stream, self.device)))

    def close(self):
        if getattr(self, "_h", None):
            nat.lib().tt_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_TUNED = {}


def _problem_key(problems, precision):
    import hashlib
    txt = repr((precision, [(tuple(p["dims"]), tuple(tuple(r) for r in p["summand_ranks"]), tuple(p["ells"]),
                             float(p.get("tol", 0.0))) for p in problems]))
    return hashlib.sha1(txt.encode()).hexdigest()


def tune_batch_schedule(problems, batch, *, precision="mixed", widths=(1, 2, 4), qr_ctas=(4, 8, 16), reps=2,
                        cache_path=None, stream=None):
    """Autotuner of the batched schedule: captures the batch for every
    (width, qr_ctas) candidate of the fused grouped-launch schedule, times
    `reps` replays with CUDA events and returns ((width, qr_ctas), {candidate:
    ms}). The choice is cached per problem set (sha1 of the shapes, ranks and
    precision) in this process and, with cache_path, in that JSON file."""
    import json
    import os
    key = _problem_key(problems, precision)
    if key in _TUNED:
        return _TUNED[key]
    if cache_path and os.path.exists(cache_path):
        try:
            db = json.load(open(cache_path))
            if key in db:
                best = tuple(db[key]["best"])
                _TUNED[key] = (best, {tuple(map(int, k.split(","))): v for k, v in db[key]["ms"].items()})
                return _TUNED[key]
        except (ValueError, KeyError, OSError):
            pass
    B = len(problems)
    times = {}
    for w in sorted({max(1, min(int(c), B)) for c in widths}):
        for q in sorted({int(c) for c in qr_ctas}):
            plan = BatchRoundingPlan(problems, precision=precision, width=w, qr_ctas=q)
            plan(batch)                                   # warm-up replay
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                plan(batch)
            e1.record()
            torch.cuda.synchronize()
            times[(w, q)] = e0.elapsed_time(e1) / reps
            plan.close()
    best = min(times, key=times.get)
    _TUNED[key] = (best, times)
    if cache_path:
        try:
            db = json.load(open(cache_path)) if os.path.exists(cache_path) else {}
        except (ValueError, OSError):
            db = {}
        db[key] = {"best": list(best), "ms": {f"{w},{q}": t for (w, q), t in times.items()}}
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        json.dump(db, open(cache_path, "w"), indent=1)
    return _TUNED[key]


def tune_batch_width(problems, batch, *, precision="mixed", candidates=(1, 2, 4), reps=2, stream=None):
    """tune_batch_schedule over the width only (qr_ctas = 8): (best width, {width: ms})."""
    (w, _), times = tune_batch_schedule(problems, batch, precision=precision, widths=candidates, qr_ctas=(8,),
                                        reps=reps, stream=stream)
    return w, {k[0]: v for k, v in times.items()}


def _sum_args(summands):
    N = len(summands[0])
    dims = [int(c.shape[1]) for c in summands[0]]
    ranks = []
    for j, Y in enumerate(summands):
        if len(Y) != N:
            raise ValueError("all summands need the same order")
        ranks += [int(Y[0].shape[0])] + [int(c.shape[2]) for c in Y]
        for n, c in enumerate(Y):
            _check_core(c, f"summand {j} core {n}")
            if int(c.shape[1]) != dims[n]:
                raise ValueError("mode sizes differ between summands")
    flat = [c for Y in summands for c in Y]
    return N, len(summands), dims, ranks, flat


def _workspace(nbytes, device, workspace):
    if workspace is None:
        workspace = torch.empty(max(int(nbytes), 1) + 256, dtype=torch.uint8, device=device)
    p = workspace.data_ptr()
    p += (-p) % 256
    return workspace, ctypes.c_void_p(p), workspace.numel() - (p - workspace.data_ptr())


def tt_round_det(summands, *, tol=0.0, max_rank=0, coeffs=None, workspace=None, stream=None):
    """Algorithms 1 + 2 (deterministic TT-SVD rounding) of the formed sum."""
    N, K, dims, ranks, flat = _sum_args(summands)
    device = summands[0][0].device
    L = nat.lib()
    dims_a, ranks_a = _i64(dims), _i64(ranks)
    caps = (ctypes.c_int64 * N)()
    _check(L.tt_round_det_out_capacity(N, K, dims_a, ranks_a, caps))
    out = [torch.empty(int(caps[n]), dtype=torch.float64, device=device) for n in range(N)]
    nb = L.tt_round_det_workspace(N, K, dims_a, ranks_a, float(tol), int(max_rank))
    if nb == 0:
        raise TTError(1, nat.last_error())
    workspace, wp, wb = _workspace(nb, device, workspace)
    co = (ctypes.c_double * K)(*[float(c) for c in coeffs]) if coeffs is not None else None
    out_ranks = (ctypes.c_int64 * (N + 1))()
    _check(L.tt_round_det(N, K, dims_a, ranks_a, _ptrs(flat), co, float(tol), int(max_rank), _ptrs(out), out_ranks,
                          wp, wb, _stream(stream, device)))
    r = [int(x) for x in out_ranks]
    return [out[n][:r[n] * dims[n] * r[n + 1]].view(r[n], dims[n], r[n + 1]) for n in range(N)]


def tt_orthrand_omega_ranks(dims, ranks_per_summand):
    N = len(dims)
    K = len(ranks_per_summand)
    flat = [int(r) for R in ranks_per_summand for r in R]
    rp = (ctypes.c_int64 * (N + 1))()
    _check(nat.lib().tt_orthrand_omega_ranks(N, K, _i64(dims), _i64(flat), rp))
    return [int(x) for x in rp]


def tt_round_orthrand(summands, ells, *, omega=None, seed=0, coeffs=None, workspace=None, stream=None):
    """Algorithm 4 (Orthogonalize-then-Randomize) of the formed sum.
    omega: optional list of N-1 Gaussian matrices Omega_n (R'_n x l_n)."""
    N, K, dims, ranks, flat = _sum_args(summands)
    device = summands[0][0].device
    ell = clamp_ranks(dims, ells)
    L = nat.lib()
    dims_a, ranks_a, ell_a = _i64(dims), _i64(ranks), _i64(ell)
    om = None
    if omega is not None:
        rp = tt_orthrand_omega_ranks(dims, [ranks[j * (N + 1):(j + 1) * (N + 1)] for j in range(K)])
        for n in range(1, N):
            o = omega[n - 1]
            if not (o.is_cuda and o.dtype == torch.float64 and o.is_contiguous() and tuple(o.shape) == (rp[n], ell[n])):
                raise ValueError(f"omega[{n - 1}] must be a contiguous float64 CUDA ({rp[n]}, {ell[n]}) matrix")
        om = _ptrs(list(omega) + [omega[0]])
    out = [torch.empty((ell[n], dims[n], ell[n + 1]), dtype=torch.float64, device=device) for n in range(N)]
    nb = L.tt_round_orthrand_workspace(N, K, dims_a, ranks_a, ell_a)
    if nb == 0:
        raise TTError(1, nat.last_error())
    workspace, wp, wb = _workspace(nb, device, workspace)
    co = (ctypes.c_double * K)(*[float(c) for c in coeffs]) if coeffs is not None else None
    out_ranks = (ctypes.c_int64 * (N + 1))()
    _check(L.tt_round_orthrand(N, K, dims_a, ranks_a, _ptrs(flat), co, ell_a, om, ctypes.c_uint64(int(seed)),
                               _ptrs(out), out_ranks, wp, wb, _stream(stream, device)))
    return out


def tt_round_twosided(summands, ells, *, rhos=None, sketch_left=None, sketch_right=None, seed=0, coeffs=None,
                      precision="fp64", workspace=None, stream=None):
    """Algorithm 6 (Two-Sided-Randomization) of a sum without forming it
    (precision "fp64", or "mixed": contractions as emulated FP64 products on
    the tensor cores)."""
    import math
    N, K, dims, ranks, flat = _sum_args(summands)
    device = summands[0][0].device
    ell = clamp_ranks(dims, ells)
    rr = clamp_ranks(dims, rhos if rhos is not None else [int(math.ceil(1.5 * x)) for x in ell])
    L = nat.lib()
    dims_a, ranks_a, ell_a, rho_a = _i64(dims), _i64(ranks), _i64(ell), _i64(rr)
    for sk, rk, name in ((sketch_left, ell, "sketch_left"), (sketch_right, rr, "sketch_right")):
        if sk is not None:
            for n, c in enumerate(sk):
                _check_core(c, f"{name} core {n}")
                if tuple(c.shape) != (rk[n], dims[n], rk[n + 1]):
                    raise ValueError(f"{name} core {n} has shape {tuple(c.shape)}")
    out = [torch.empty((ell[n], dims[n], ell[n + 1]), dtype=torch.float64, device=device) for n in range(N)]
    nb = L.tt_round_twosided_workspace(N, K, dims_a, ranks_a, ell_a, rho_a, _PREC[precision])
    if nb == 0:
        raise TTError(1, nat.last_error())
    workspace, wp, wb = _workspace(nb, device, workspace)
    co = (ctypes.c_double * K)(*[float(c) for c in coeffs]) if coeffs is not None else None
    out_ranks = (ctypes.c_int64 * (N + 1))()
    _check(L.tt_round_twosided(N, K, dims_a, ranks_a, _ptrs(flat), co, ell_a, rho_a,
                               _ptrs(sketch_left) if sketch_left is not None else None,
                               _ptrs(sketch_right) if sketch_right is not None else None,
                               ctypes.c_uint64(int(seed)), _PREC[precision], _ptrs(out), out_ranks, wp, wb,
                               _stream(stream, device)))
    return out


def tt_round_twosided_orth(summands, ells, *, rhos=None, sketch_left=None, sketch_right=None, seed=0, coeffs=None,
                           tol=0.0, precision="fp64", workspace=None, stream=None):
    """Algorithm 6 with the orthogonalizing restructure: the same tensor as
    tt_round_twosided in left-orthogonal form, truncated to tol (Section 3.2)
    when tol > 0. Returns the cores at the decided ranks."""
    import math
    N, K, dims, ranks, flat = _sum_args(summands)
    device = summands[0][0].device
    ell = clamp_ranks(dims, ells)
    rr = clamp_ranks(dims, rhos if rhos is not None else [int(math.ceil(1.5 * x)) for x in ell])
    L = nat.lib()
    dims_a, ranks_a, ell_a, rho_a = _i64(dims), _i64(ranks), _i64(ell), _i64(rr)
    for sk, rk, name in ((sketch_left, ell, "sketch_left"), (sketch_right, rr, "sketch_right")):
        if sk is not None:
            for n, c in enumerate(sk):
                _check_core(c, f"{name} core {n}")
                if tuple(c.shape) != (rk[n], dims[n], rk[n + 1]):
                    raise ValueError(f"{name} core {n} has shape {tuple(c.shape)}")
    out = [torch.empty((ell[n], dims[n], ell[n + 1]), dtype=torch.float64, device=device) for n in range(N)]
    nb = L.tt_round_twosided_orth_workspace(N, K, dims_a, ranks_a, ell_a, rho_a, float(tol), _PREC[precision])
    if nb == 0:
        raise TTError(1, nat.last_error())
    workspace, wp, wb = _workspace(nb, device, workspace)
    co = (ctypes.c_double * K)(*[float(c) for c in coeffs]) if coeffs is not None else None
    out_ranks = (ctypes.c_int64 * (N + 1))()
    _check(L.tt_round_twosided_orth(N, K, dims_a, ranks_a, _ptrs(flat), co, ell_a, rho_a,
                                    _ptrs(sketch_left) if sketch_left is not None else None,
                                    _ptrs(sketch_right) if sketch_right is not None else None,
                                    ctypes.c_uint64(int(seed)), float(tol), _PREC[precision], _ptrs(out), out_ranks,
                                    wp, wb, _stream(stream, device)))
    r = [int(x) for x in out_ranks]
    return [out[n].view(-1)[:r[n] * dims[n] * r[n + 1]].view(r[n], dims[n], r[n + 1]) for n in range(N)]


def tt_truncate_lorth(cores, *, tol=0.0, max_rank=0, workspace=None, stream=None):
    """Section 3.2 truncation of a left-orthogonal TT (list of float64 CUDA
    cores). The cores are copied first (the call works in place on the copy);
    returns the truncated cores."""
    N = len(cores)
    device = cores[0].device
    dims = [int(c.shape[1]) for c in cores]
    ranks = [int(cores[0].shape[0])] + [int(c.shape[2]) for c in cores]
    work = []
    for n, c in enumerate(cores):
        _check_core(c, f"core {n}")
        work.append(c.clone())
    L = nat.lib()
    dims_a, ranks_a = _i64(dims), _i64(ranks)
    nb = L.tt_truncate_lorth_workspace(N, dims_a, ranks_a, float(tol), int(max_rank))
    if nb == 0:
        raise TTError(1, nat.last_error())
    workspace, wp, wb = _workspace(nb, device, workspace)
    out_ranks = (ctypes.c_int64 * (N + 1))()
    _check(L.tt_truncate_lorth(N, dims_a, ranks_a, _ptrs(work), float(tol), int(max_rank), out_ranks, wp, wb,
                               _stream(stream, device)))
    r = [int(x) for x in out_ranks]
    return [work[n].view(-1)[:r[n] * dims[n] * r[n + 1]].view(r[n], dims[n], r[n + 1]) for n in range(N)]


def _tt_args(cores, name="core"):
    dims = [int(c.shape[1]) for c in cores]
    ranks = [int(cores[0].shape[0])] + [int(c.shape[2]) for c in cores]
    for n, c in enumerate(cores):
        _check_core(c, f"{name} {n}")
    return dims, ranks


def tt_inner(X, Ys, *, workspace=None, stream=None):
    """<X, Y_j> for every TT in Ys (Algorithm 3 run to the first core), as a
    float64 CUDA tensor of len(Ys) values."""
    N = len(X)
    device = X[0].device
    dims, rx = _tt_args(X, "X core")
    N2, K, dims2, ranks, flat = _sum_args(Ys)
    if N2 != N or dims2 != dims:
        raise ValueError("X and Ys need the same order and mode sizes")
    L = nat.lib()
    out = torch.empty(K, dtype=torch.float64, device=device)
    nb = L.tt_inner_workspace(N, _i64(dims), _i64(rx), K, _i64(ranks))
    if nb == 0:
        raise TTError(1, nat.last_error())
    workspace, wp, wb = _workspace(nb, device, workspace)
    _check(L.tt_inner(N, _i64(dims), _i64(rx), _ptrs(X), K, _i64(ranks), _ptrs(flat), ctypes.c_void_p(out.data_ptr()),
                      wp, wb, _stream(stream, device)))
    return out


def tt_norm(X, *, workspace=None, stream=None):
    """||X|| (float64 CUDA scalar tensor)."""
    N = len(X)
    device = X[0].device
    dims, r = _tt_args(X)
    L = nat.lib()
    out = torch.empty(1, dtype=torch.float64, device=device)
    nb = L.tt_norm_workspace(N, _i64(dims), _i64(r))
    if nb == 0:
        raise TTError(1, nat.last_error())
    workspace, wp, wb = _workspace(nb, device, workspace)
    _check(L.tt_norm(N, _i64(dims), _i64(r), _ptrs(X), ctypes.c_void_p(out.data_ptr()), wp, wb,
                     _stream(stream, device)))
    return out[0]


def tt_mode_products(mats, cores, *, workspace=None, stream=None):
    """[A_q x_2 core_q for q]: out_q(a, j, b) = sum_i A_q(j, i) core_q(a, i, b)
    for float64 CUDA matrices A_q (J x I) and cores (r0, I, r1), one grouped launch."""
    if len(mats) != len(cores):
        raise ValueError("one matrix per core")
    if not cores:
        return []
    device = cores[0].device
    shapes, outs, amats = [], [], []
    for q, (A, c) in enumerate(zip(mats, cores)):
        _check_core(c, f"core {q}")
        if not (A.is_cuda and A.dtype == torch.float64 and A.dim() == 2 and A.shape[1] == c.shape[1]):
            raise ValueError(f"matrix {q}: expected a float64 CUDA (J, I) matrix with I = {c.shape[1]}")
        A = A.contiguous()
        amats.append(A)
        shapes += [int(c.shape[0]), int(c.shape[1]), int(c.shape[2]), int(A.shape[0])]
        outs.append(torch.empty((int(c.shape[0]), int(A.shape[0]), int(c.shape[2])), dtype=torch.float64,
                                device=device))
    L = nat.lib()
    nb = L.tt_mode_products_workspace(len(cores), _i64(shapes))
    if nb == 0:
        raise TTError(1, nat.last_error())
    workspace, wp, wb = _workspace(nb, device, workspace)
    _check(L.tt_mode_products(len(cores), _i64(shapes), _ptrs(amats), _ptrs(cores), _ptrs(outs), wp, wb,
                              _stream(stream, device)))
    return outs


def tt_round_gram_schmidt(W, basis, ells, *, tol=0.0, sketch=None, seed=0, precision="fp64", workspace=None,
                          stream=None):
    """One Gram-Schmidt step of TT-GMRES (Section 4.2) in one call:
    h_j = <V_j, W>, Z = round(W - sum_j h_j V_j), V_new = Z / ||Z||.
    Returns (V_new cores, h as a list of k + 1 floats: h_1..h_k, ||Z||)."""
    N = len(W)
    device = W[0].device
    dims, rw = _tt_args(W, "W core")
    k = len(basis)
    rv, fv = [], []
    for j, V in enumerate(basis):
        d, r = _tt_args(V, f"basis {j} core")
        if d != dims:
            raise ValueError("basis tensors need the mode sizes of W")
        rv += r
        fv += list(V)
    ell = clamp_ranks(dims, ells)
    out = [torch.empty((ell[n], dims[n], ell[n + 1]), dtype=torch.float64, device=device) for n in range(N)]
    sk_arr = None
    if sketch is not None:
        for n, c in enumerate(sketch):
            _check_core(c, f"sketch core {n}")
        sk_arr = _ptrs(sketch)
    L = nat.lib()
    prec = _PREC[precision]
    nb = L.tt_round_gram_schmidt_workspace(N, _i64(dims), _i64(rw), k, _i64(rv), _i64(ell), float(tol), prec)
    if nb == 0:
        raise TTError(1, nat.last_error())
    workspace, wp, wb = _workspace(nb, device, workspace)
    out_ranks = (ctypes.c_int64 * (N + 1))()
    h = (ctypes.c_double * (k + 1))()
    _check(L.tt_round_gram_schmidt(N, _i64(dims), _i64(rw), _ptrs(W), k, _i64(rv), _ptrs(fv) if k else None,
                                   _i64(ell), sk_arr, ctypes.c_uint64(int(seed)), float(tol), prec, _ptrs(out),
                                   out_ranks, h, wp, wb, _stream(stream, device)))
    r = [int(x) for x in out_ranks]
    Vn = [out[n].view(-1)[:r[n] * dims[n] * r[n + 1]].view(r[n], dims[n], r[n + 1]) for n in range(N)]
    return Vn, [float(x) for x in h]


def _round_rand_f32(Y, ells, *, tol=0.0, sketch=None, seed=0, precision="mixed", workspace=None, stream=None):
    N = len(Y)
    device = Y[0].device
    dims = [int(c.shape[1]) for c in Y]
    ranks = [int(Y[0].shape[0])] + [int(c.shape[2]) for c in Y]
    for n, c in enumerate(Y):
        _check_core(c, f"core {n}", torch.float32)
    ell = clamp_ranks(dims, ells)
    sk_arr = None
    if sketch is not None:
        for n in range(1, N):
            _check_core(sketch[n], f"sketch core {n}", torch.float32)
            if tuple(sketch[n].shape) != (ell[n], dims[n], ell[n + 1]):
                raise ValueError(f"sketch core {n} has shape {tuple(sketch[n].shape)}")
        sk_arr = _ptrs([sketch[n] if n > 0 else Y[0] for n in range(N)])
    out = [torch.empty((ell[n], dims[n], ell[n + 1]), dtype=torch.float32, device=device) for n in range(N)]
    L = nat.lib()
    prec = _PREC[precision]
    nb = L.tt_round_rand_f32_workspace(N, _i64(dims), _i64(ranks), _i64(ell), float(tol), prec)
    if nb == 0:
        raise TTError(1, nat.last_error())
    workspace, wp, wb = _workspace(nb, device, workspace)
    out_ranks = (ctypes.c_int64 * (N + 1))()
    _check(L.tt_round_rand_f32(N, _i64(dims), _i64(ranks), _ptrs(Y), _i64(ell), sk_arr, ctypes.c_uint64(int(seed)),
                               float(tol), prec, _ptrs(out), out_ranks, wp, wb, _stream(stream, device)))
    r = [int(x) for x in out_ranks]
    return [out[n].view(-1)[:r[n] * dims[n] * r[n + 1]].view(r[n], dims[n], r[n + 1]) for n in range(N)]


def tt_round_rand(Y, ells, **kw):
    """Algorithm 5 (single TT, Randomize-then-Orthogonalize): tt_round_sum_rand
    with K = 1. float32 cores take the float32 entry point (precision
    "mixed" by default: FP32-class tensor-core contractions, FP64 QR)."""
    if kw.get("coeffs") is not None:
        raise ValueError("tt_round_rand takes no coefficients")
    if Y[0].dtype == torch.float32:
        kw.setdefault("precision", "mixed")
        return _round_rand_f32(Y, ells, **kw)
    return tt_round_sum_rand([Y], ells, **kw)


TT_ESINGULAR = 5
TT_ETIMEOUT = 6
DEV_TIMEOUT = 1
DEV_QR_FAIL = 2


def debug_inject_device_status(bits):
    """Test hook: the next read-back of a device status word sees `bits`
    (DEV_TIMEOUT, DEV_QR_FAIL), written over the device word by a host copy."""
    nat.lib().tt_debug_inject_device_status(int(bits))


QR_AUTO, QR_CHAIN, QR_FORCE_FALLBACK, QR_COOP_THEN_FALLBACK = 0, 1, 2, 3


def set_qr_mode(mode):
    """How later calls run their thin QRs: QR_AUTO (one cooperative launch
    where it fits), QR_CHAIN (one launch per Cholesky-QR pass) or
    QR_FORCE_FALLBACK (Householder TSQR for every QR with k <= 96) or
    QR_COOP_THEN_FALLBACK (testing: the cooperative chain, then the fallback as
    after a breakdown)."""
    _check(nat.lib().tt_set_qr_mode(int(mode)))


GEMM_AUTO, GEMM_THREE_PASS, GEMM_FUSED = 0, 1, 2


def set_gemm_mode(mode):
    """GEMM_AUTO (fused for groups with large digit planes), GEMM_THREE_PASS or
    GEMM_FUSED; bit-identical results."""
    _check(nat.lib().tt_set_gemm_mode(int(mode)))


def tsqr_fallback_runs():
    """Householder fallback QRs run on the current device since the library loaded."""
    v = ctypes.c_int64()
    _check(nat.lib().tt_tsqr_fallback_runs(ctypes.byref(v)))
    return int(v.value)


def probe_fp64_rate(iters=1 << 16, stream=None):
    """Measured FP64 FMA rate of the current GPU (TFLOP/s), from a register-only FMA loop."""
    v = ctypes.c_double()
    dev = torch.device("cuda", torch.cuda.current_device())
    _check(nat.lib().tt_probe_fp64_rate(int(iters), ctypes.byref(v), _stream(stream, dev)))
    return float(v.value)


def probe_pivot_rsqrt(n=1 << 22, stream=None):
    """(max ulp distance, points that differ) of the QR pivots' reciprocal
    square root against CUDA's rsqrt over n points of the normal range."""
    mu, nd = ctypes.c_int64(), ctypes.c_int64()
    dev = torch.device("cuda", torch.cuda.current_device())
    _check(nat.lib().tt_probe_pivot_rsqrt(int(n), ctypes.byref(mu), ctypes.byref(nd), _stream(stream, dev)))
    return int(mu.value), int(nd.value)


def prof_enable(on=True):
    _check(nat.lib().tt_prof_enable(1 if on else 0))


def prof_reset():
    _check(nat.lib().tt_prof_reset())


def prof_read_kind(kind):
    """(ms, flops, launches) of one kind of timed launch: 0 contraction groups, 1 QR passes."""
    ms, fl, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    _check(nat.lib().tt_prof_read_kind(int(kind), ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(n)))
    return ms.value, fl.value, n.value


def prof_read():
    """(gemm_ms, gemm_flops, gemm_launches, kernel_launches) since the last reset."""
    ms, fl = ctypes.c_double(), ctypes.c_double()
    gl, kl = ctypes.c_int64(), ctypes.c_int64()
    _check(nat.lib().tt_prof_read(ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(gl), ctypes.byref(kl)))
    return ms.value, fl.value, gl.value, kl.value
