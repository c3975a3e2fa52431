"""Thin Python binding of the C ABI in include/smc.h (ctypes).

Argument marshalling only: every step of the SMC path runs in libsmc.so's
CUDA kernels.  PyTorch supplies the device workspace and the stream.  The
binding fails loudly when the library is missing; there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsmc.so")

OK, E_ARG, E_WORKSPACE, E_NONFINITE, E_TIMEOUT, E_CUDA, E_STATE, E_RANGE = range(8)
MULTINOMIAL, STRATIFIED, SYSTEMATIC, RESIDUAL = range(4)
SCHEMES = {"multinomial": MULTINOMIAL, "stratified": STRATIFIED, "systematic": SYSTEMATIC,
           "residual": RESIDUAL, "residual_systematic": RESIDUAL + 1, "residual_stratified": RESIDUAL + 2}
MODEL_CV, MODEL_CV_GAUSS, MODEL_GMM = range(3)
ALPHA_LINEAR, ALPHA_PRIOR, ALPHA_ADAPTIVE = range(3)
GMM_RW, GMM_MALA, GMM_RW_MALA = range(3)


class CVParams(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("sd_pos", ctypes.c_double), ("sd_vel", ctypes.c_double),
                ("obs_scale", ctypes.c_double), ("obs_df", ctypes.c_double), ("sd_pos0", ctypes.c_double),
                ("sd_vel0", ctypes.c_double)]


class GMMParams(ctypes.Structure):
    _fields_ = [("n_comp", ctypes.c_int32), ("schedule", ctypes.c_int32), ("n_iter", ctypes.c_int32),
                ("shape0", ctypes.c_int32), ("power", ctypes.c_double), ("mu0", ctypes.c_double),
                ("sd0", ctypes.c_double), ("rate0", ctypes.c_double), ("move", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("mala_step", ctypes.c_double), ("ess_target", ctypes.c_double)]


class Config(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("precision", ctypes.c_int32), ("n_particles", ctypes.c_int64),
                ("max_records", ctypes.c_int32), ("scheme", ctypes.c_int32), ("threshold", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("stream_id", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("max_data", ctypes.c_int64), ("cv", CVParams), ("gmm", GMMParams),
                ("checkpoint_every", ctypes.c_int32), ("reserved2", ctypes.c_int32)]


class Record(ctypes.Structure):
    _fields_ = [("log_norm", ctypes.c_double), ("log_evidence", ctypes.c_double), ("ess", ctypes.c_double),
                ("mean", ctypes.c_double * 2), ("max_lw", ctypes.c_double), ("path_u", ctypes.c_double),
                ("path_log_z", ctypes.c_double), ("alpha", ctypes.c_double), ("accept", ctypes.c_double * 3),
                ("t", ctypes.c_int32), ("resampled", ctypes.c_int32), ("status", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("accept_mala", ctypes.c_double), ("mean_post", ctypes.c_double * 2)]

    def as_dict(self):
        return dict(t=self.t, L=self.log_norm, logZ=self.log_evidence, ess=self.ess, mean_x=self.mean[0],
                    mean_y=self.mean[1], max_lw=self.max_lw, path_u=self.path_u, path_log_z=self.path_log_z,
                    alpha=self.alpha, accept=tuple(self.accept), accept_mala=self.accept_mala,
                    resampled=bool(self.resampled), status=self.status, post_mean_x=self.mean_post[0],
                    post_mean_y=self.mean_post[1])


_P = ctypes.c_void_p
_I = ctypes.c_int
_SIGS = {
    "smc_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(Config)]),
    "smc_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(Config), _P, ctypes.c_size_t, _P]),
    "smc_destroy": (_I, [_P]),
    "smc_set_data": (_I, [_P, _P, ctypes.c_int64, _I]),
    "smc_initialize": (_I, [_P]),
    "smc_move": (_I, [_P]),
    "smc_resample": (_I, [_P, _I]),
    "smc_mcmc": (_I, [_P]),
    "smc_iterate": (_I, [_P, ctypes.c_int32]),
    "smc_iterate_host": (_I, [_P, _P, ctypes.POINTER(Record)]),
    "smc_add_log_weight": (_I, [_P, _P, _I]),
    "smc_ess": (_I, [_P, ctypes.POINTER(ctypes.c_double)]),
    "smc_log_evidence": (_I, [_P, ctypes.POINTER(ctypes.c_double)]),
    "smc_path_sampling": (_I, [_P, ctypes.POINTER(ctypes.c_double)]),
    "smc_iteration": (_I, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "smc_state_dim": (_I, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "smc_read_state": (_I, [_P, _P, _I]),
    "smc_read_log_weight": (_I, [_P, _P, _I]),
    "smc_read_ancestors": (_I, [_P, _P, _I]),
    "smc_read_cdf": (_I, [_P, _P, _I]),
    "smc_read_history": (_I, [_P, ctypes.POINTER(Record), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "smc_write_state": (_I, [_P, _P, _I]),
    "smc_write_log_weight": (_I, [_P, _P, _I]),
    "smc_sync": (_I, [_P]),
    "smc_set_move_events": (_I, [_P, _P, _P]),
    "smc_checkpoint": (_I, [_P, _P, ctypes.POINTER(ctypes.c_size_t)]),
    "smc_gmm_log_target": (_I, [_P, _P, ctypes.c_int64, ctypes.c_double, _P, _P]),
    "smc_restore": (_I, [_P, _P, ctypes.c_size_t]),
    "smc_error_string": (ctypes.c_char_p, [_I]),
    "smc_philox4x32_10": (_I, [_P, ctypes.POINTER(ctypes.c_uint32), _P, ctypes.c_int64, _P]),
    "smc_pf_grad": (_I, [_P, _P]),
    "smc_pf_replay": (_I, [_P, _P, ctypes.POINTER(ctypes.c_double)]),
    "smc_read_ancestor_history": (_I, [_P, ctypes.c_int32, _P, _I]),
    "smc_resample_systematic_noalloc": (_I, [_P, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32,
                                             _P, _P]),
    "smc_resample_noalloc_status": (_I, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "smc_set_wait_limit": (_I, [ctypes.c_uint32]),
    "smc_shard_configure": (_I, [_P, ctypes.c_int64, ctypes.c_int64]),
    "smc_shard_move": (_I, [_P, _P]),
    "smc_shard_finalize": (_I, [_P, _P, ctypes.c_int32]),
    "smc_shard_total": (_I, [_P, _P]),
    "smc_shard_select": (_I, [_P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P]),
    "smc_shard_pack": (_I, [_P, _P, ctypes.c_int64, ctypes.c_int64, _P]),
    "smc_shard_unpack": (_I, [_P, _P]),
    "smc_shard_mcmc": (_I, [_P, _P]),
    "smc_shard_mcmc_finalize": (_I, [_P, _P, ctypes.c_int32]),
    "smc_mufu_rate": (_I, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double)]),
    "smc_wait_selftest": (_I, [_P]),
    "smc_batch_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(Config), _P, _P, ctypes.c_int32]),
    "smc_batch_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(Config), _P, _P, ctypes.c_int32, _P,
                              ctypes.c_size_t, _P]),
    "smc_batch_destroy": (_I, [_P]),
    "smc_batch_set_streams": (_I, [_P, _P]),
    "smc_batch_set_data": (_I, [_P, ctypes.c_int32, _P, _I]),
    "smc_batch_initialize": (_I, [_P]),
    "smc_batch_iterate": (_I, [_P, ctypes.c_int32]),
    "smc_batch_run": (_I, [_P]),
    "smc_batch_tune": (_I, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "smc_batch_log_evidence": (_I, [_P, _P]),
    "smc_batch_read_history": (_I, [_P, ctypes.c_int32, ctypes.POINTER(Record), ctypes.c_int32,
                                    ctypes.POINTER(ctypes.c_int32)]),
    "smc_batch_read_state": (_I, [_P, ctypes.c_int32, _P, _I]),
}

_lib = None


def lib():
    """The loaded libsmc.so (raises when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is missing: run __graft_entry__.build() (nvcc, sm_103a)")
        L = ctypes.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class SMCError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = lib().smc_error_string(code).decode()
        super().__init__(f"{where}: {msg} (code {code})")


def check(code, where):
    if code != OK:
        raise SMCError(code, where)


FLAG_KEEP_CDF = 1
FLAG_RECORD = 2
FLAG_POST_MEAN = 4
FLAG_INPLACE = 8


def make_config(model="cv", n=1024, precision=32, scheme="systematic", threshold=0.5, seed=0, stream_id=0,
                max_records=None, max_data=1000, cv=None, gmm=None, keep_cdf=True, record=False,
                checkpoint_every=16, post_mean=False, inplace=False):
    c = Config()
    c.model = {"cv": MODEL_CV, "cv_gauss": MODEL_CV_GAUSS, "gmm": MODEL_GMM}[model]
    c.precision = precision
    c.n_particles = int(n)
    c.scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    c.threshold = float(threshold)
    c.seed = int(seed)
    c.stream_id = int(stream_id)
    c.flags = ((FLAG_KEEP_CDF if keep_cdf else 0) | (FLAG_RECORD if record else 0)
               | (FLAG_POST_MEAN if post_mean else 0) | (FLAG_INPLACE if inplace else 0))
    c.checkpoint_every = int(checkpoint_every)
    c.max_data = int(max_data)
    c.max_records = int(max_records if max_records is not None else max(2, max_data + 1))
    p = dict(delta=0.1, sd_pos=0.02, sd_vel=1.0, obs_scale=0.5, obs_df=10.0, sd_pos0=1.0, sd_vel0=1.0)
    p.update(cv or {})
    for k, v in p.items():
        setattr(c.cv, k, float(v))
    g = dict(n_comp=4, schedule=ALPHA_PRIOR, n_iter=500, shape0=1, power=5.0, mu0=0.0, sd0=10.0, rate0=1.0,
             move=GMM_RW, mala_step=0.05, ess_target=0.5)
    g.update(gmm or {})
    for k, v in g.items():
        setattr(c.gmm, k, v)
    return c


class Sampler:
    """One SMC context on the current CUDA device (Sampler<T> of the paper).

    The workspace is a torch uint8 tensor; `stream` a torch.cuda.Stream (or
    None for torch's current stream).
    """

    def __init__(self, config, stream=None, device=None):
        import torch
        self.torch = torch
        self.cfg = config
        self.device = torch.device(device or "cuda")
        L = lib()
        nbytes = L.smc_workspace_bytes(ctypes.byref(config))
        if nbytes == 0:
            raise SMCError(E_ARG, "smc_workspace_bytes")
        self.nbytes = nbytes
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        self.ws_ptr = (base + 255) & ~255
        self.ctx = _P()
        check(L.smc_create(ctypes.byref(self.ctx), ctypes.byref(config), _P(self.ws_ptr), nbytes,
                           _P(self.stream.cuda_stream)), "smc_create")
        d = ctypes.c_int32()
        check(L.smc_state_dim(self.ctx, ctypes.byref(d)), "smc_state_dim")
        self.dim = d.value
        self.n = config.n_particles
        self.rdtype = np.float32 if config.precision == 32 else np.float64
        self.tdtype = torch.float32 if config.precision == 32 else torch.float64

    def close(self):
        if self.ctx:
            lib().smc_destroy(self.ctx)
            self.ctx = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the paper's sampler decomposition --
    def set_data(self, obs):
        a = np.ascontiguousarray(np.asarray(obs, dtype=np.float64))
        count = a.shape[0]
        check(lib().smc_set_data(self.ctx, a.ctypes.data_as(_P), count, 0), "smc_set_data")

    def set_data_device(self, obs_tensor):
        """Observations already on the device (float64, contiguous)."""
        assert obs_tensor.dtype == self.torch.float64 and obs_tensor.is_contiguous()
        check(lib().smc_set_data(self.ctx, _P(obs_tensor.data_ptr()), obs_tensor.shape[0], 1), "smc_set_data")

    def initialize(self):
        check(lib().smc_initialize(self.ctx), "smc_initialize")

    def move(self):
        check(lib().smc_move(self.ctx), "smc_move")

    def resample(self, force=False):
        check(lib().smc_resample(self.ctx, 1 if force else 0), "smc_resample")

    def mcmc(self):
        check(lib().smc_mcmc(self.ctx), "smc_mcmc")

    def iterate(self, n=1):
        check(lib().smc_iterate(self.ctx, int(n)), "smc_iterate")

    def iterate_host(self, obs_t=None):
        rec = Record()
        if obs_t is None:
            p = None
        else:
            buf = np.ascontiguousarray(np.asarray(obs_t, dtype=np.float64))
            p = buf.ctypes.data_as(_P)
        check(lib().smc_iterate_host(self.ctx, p, ctypes.byref(rec)), "smc_iterate_host")
        return rec

    def sync(self):
        check(lib().smc_sync(self.ctx), "smc_sync")

    def wait_selftest(self):
        check(lib().smc_wait_selftest(self.ctx), "smc_wait_selftest")

    def set_move_events(self, before=None, after=None):
        """Record two torch.cuda.Event objects (created with timing) around
        the move kernel inside the iteration graph (None, None clears)."""
        def handle(e):
            if e is None:
                return None
            if not e.cuda_event:  # torch creates the event at its first record
                e.record()
            return ctypes.c_void_p(e.cuda_event)
        check(lib().smc_set_move_events(self.ctx, handle(before), handle(after)), "smc_set_move_events")

    def ess(self):
        v = ctypes.c_double()
        check(lib().smc_ess(self.ctx, ctypes.byref(v)), "smc_ess")
        return v.value

    def log_evidence(self):
        v = ctypes.c_double()
        check(lib().smc_log_evidence(self.ctx, ctypes.byref(v)), "smc_log_evidence")
        return v.value

    def path_sampling(self):
        v = ctypes.c_double()
        check(lib().smc_path_sampling(self.ctx, ctypes.byref(v)), "smc_path_sampling")
        return v.value

    def iteration(self):
        v = ctypes.c_int32()
        check(lib().smc_iteration(self.ctx, ctypes.byref(v)), "smc_iteration")
        return v.value

    # -- readers (host numpy copies) --
    def state(self):
        out = np.empty((self.dim, self.n), dtype=self.rdtype)
        check(lib().smc_read_state(self.ctx, out.ctypes.data_as(_P), 0), "smc_read_state")
        return out

    def log_weight(self):
        out = np.empty(self.n, dtype=self.rdtype)
        check(lib().smc_read_log_weight(self.ctx, out.ctypes.data_as(_P), 0), "smc_read_log_weight")
        return out

    def ancestors(self):
        out = np.empty(self.n, dtype=np.int32)
        check(lib().smc_read_ancestors(self.ctx, out.ctypes.data_as(_P), 0), "smc_read_ancestors")
        return out

    def cdf(self):
        out = np.empty(self.n, dtype=np.uint64)
        check(lib().smc_read_cdf(self.ctx, out.ctypes.data_as(_P), 0), "smc_read_cdf")
        return out

    # -- readers into device tensors (the same layouts, copied on the device) --
    def read_device(self, what):
        """A new device tensor holding the context's current `what`:
        "state" (d x N), "log_weight" (N), "ancestors" (N int32) or "cdf"
        (N fixed-point values, as int64 bit patterns: every value is below
        2^62).  Only the device-to-device copy of smc_read_* runs; nothing
        crosses to the host."""
        torch = self.torch
        shape, dtype, fn = {"state": ((self.dim, self.n), self.tdtype, "smc_read_state"),
                            "log_weight": ((self.n,), self.tdtype, "smc_read_log_weight"),
                            "ancestors": ((self.n,), torch.int32, "smc_read_ancestors"),
                            "cdf": ((self.n,), torch.int64, "smc_read_cdf")}[what]
        out = torch.empty(shape, dtype=dtype, device=self.device)
        check(getattr(lib(), fn)(self.ctx, _P(out.data_ptr()), 1), fn)
        return out

    def history(self, count):
        recs = (Record * count)()
        n = ctypes.c_int32()
        check(lib().smc_read_history(self.ctx, recs, count, ctypes.byref(n)), "smc_read_history")
        return [recs[i].as_dict() for i in range(n.value)]

    def write_state(self, x):
        a = np.ascontiguousarray(np.asarray(x, dtype=self.rdtype))
        assert a.shape == (self.dim, self.n)
        check(lib().smc_write_state(self.ctx, a.ctypes.data_as(_P), 0), "smc_write_state")

    def write_log_weight(self, lw):
        a = np.ascontiguousarray(np.asarray(lw, dtype=self.rdtype))
        assert a.shape == (self.n,)
        check(lib().smc_write_log_weight(self.ctx, a.ctypes.data_as(_P), 0), "smc_write_log_weight")

    def pf_grad(self):
        """d log Z-hat / d(sd_pos, sd_vel, obs_scale, obs_df) of the recorded run."""
        g = np.zeros(4)
        check(lib().smc_pf_grad(self.ctx, g.ctypes.data_as(_P)), "smc_pf_grad")
        return g

    def pf_replay(self, theta):
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        v = ctypes.c_double()
        check(lib().smc_pf_replay(self.ctx, th.ctypes.data_as(_P), ctypes.byref(v)), "smc_pf_replay")
        return v.value

    def ancestor_history(self, t):
        out = np.empty(self.n, dtype=np.int32)
        check(lib().smc_read_ancestor_history(self.ctx, int(t), out.ctypes.data_as(_P), 0),
              "smc_read_ancestor_history")
        return out

    def add_log_weight(self, incw):
        """lw += incw for the current iteration (normaliser, ESS, decision again)."""
        a = np.ascontiguousarray(np.asarray(incw, dtype=self.rdtype))
        assert a.shape == (self.n,)
        check(lib().smc_add_log_weight(self.ctx, a.ctypes.data_as(_P), 0), "smc_add_log_weight")

    def gmm_log_target(self, u, alpha):
        """Tempered log-target and its gradient at points u (count, 3r - 1) in
        unconstrained coordinates (a CUDA tensor of the context's precision);
        returns (log_target (count,), grad (count, 3r - 1)) as CUDA tensors."""
        torch = self.torch
        uu = u.detach().to(device=self.device, dtype=self.tdtype).t().contiguous()
        count = uu.shape[1]
        logt = torch.empty(count, dtype=self.tdtype, device=self.device)
        grad = torch.empty_like(uu)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))  # u is ready
        check(lib().smc_gmm_log_target(self.ctx, _P(uu.data_ptr()), count, float(alpha), _P(logt.data_ptr()),
                                       _P(grad.data_ptr())), "smc_gmm_log_target")
        self.sync()  # the outputs are complete on return
        return logt, grad.t()

    def checkpoint(self):
        """The complete sampler state as bytes (see smc_checkpoint)."""
        size = ctypes.c_size_t(0)
        check(lib().smc_checkpoint(self.ctx, None, ctypes.byref(size)), "smc_checkpoint")
        buf = ctypes.create_string_buffer(size.value)
        check(lib().smc_checkpoint(self.ctx, ctypes.cast(buf, _P), ctypes.byref(size)), "smc_checkpoint")
        return buf.raw[:size.value]

    def restore(self, blob):
        """Continue from a checkpoint of a sampler with the same configuration."""
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        check(lib().smc_restore(self.ctx, ctypes.cast(buf, _P), len(blob)), "smc_restore")


def mufu_rate(kind=0, blocks_per_sm=8, iters=4096):
    """(MUFU operations per second, ms) of the special-function pipe
    microbenchmark on the current device (smc_mufu_rate; kind 0 alternating
    ex2 / lg2, 1 ex2, 2 lg2)."""
    ops, ms = ctypes.c_double(), ctypes.c_double()
    check(lib().smc_mufu_rate(int(kind), int(blocks_per_sm), int(iters), ctypes.byref(ops), ctypes.byref(ms)),
          "smc_mufu_rate")
    return ops.value, ms.value


def set_wait_limit(polls):
    """Polls a bounded device wait makes before raising SMC_E_TIMEOUT on the
    current device (0: the default, 2^24)."""
    check(lib().smc_set_wait_limit(int(polls)), "smc_set_wait_limit")


def philox4x32_10(ctr, key):
    """Philox4x32-10 on the GPU through the C ABI: ctr (n, 4) uint32, key 2 uint32."""
    import torch
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    n = c.shape[0]
    dc = torch.from_numpy(c.view(np.int32)).cuda()
    do = torch.empty_like(dc)
    k = (ctypes.c_uint32 * 2)(int(key[0]), int(key[1]))
    check(lib().smc_philox4x32_10(_P(dc.data_ptr()), k, _P(do.data_ptr()), n,
                                  _P(torch.cuda.current_stream().cuda_stream)), "smc_philox4x32_10")
    torch.cuda.synchronize()
    return do.cpu().numpy().view(np.uint32)


class Batch:
    """Many independent constant-velocity filters advanced together
    (smc_batch_* of the C ABI).  n_particles and n_iter are per filter."""

    def __init__(self, config, n_particles, n_iter, stream=None, device=None):
        import torch
        self.cfg = config
        self.device = torch.device(device or "cuda")
        self.n = np.ascontiguousarray(np.asarray(n_particles, dtype=np.int64))
        self.T = np.ascontiguousarray(np.asarray(n_iter, dtype=np.int32))
        self.nf = int(self.n.shape[0])
        L = lib()
        nbytes = L.smc_batch_workspace_bytes(ctypes.byref(config), self.n.ctypes.data_as(_P),
                                             self.T.ctypes.data_as(_P), self.nf)
        if nbytes == 0:
            raise SMCError(E_ARG, "smc_batch_workspace_bytes")
        self.nbytes = nbytes
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        self.ws_ptr = (self.ws.data_ptr() + 255) & ~255
        self.ctx = _P()
        check(L.smc_batch_create(ctypes.byref(self.ctx), ctypes.byref(config), self.n.ctypes.data_as(_P),
                                 self.T.ctypes.data_as(_P), self.nf, _P(self.ws_ptr), nbytes,
                                 _P(self.stream.cuda_stream)), "smc_batch_create")
        self.rdtype = np.float32 if config.precision == 32 else np.float64

    def close(self):
        if self.ctx:
            lib().smc_batch_destroy(self.ctx)
            self.ctx = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_data(self, filter_index, obs):
        a = np.ascontiguousarray(np.asarray(obs, dtype=np.float64))
        assert a.shape == (int(self.T[filter_index]), 2)
        check(lib().smc_batch_set_data(self.ctx, int(filter_index), a.ctypes.data_as(_P), 0), "smc_batch_set_data")

    def set_streams(self, stream_ids):
        """Philox stream of each filter (smc_batch_set_streams)."""
        ids = np.ascontiguousarray(np.asarray(stream_ids, dtype=np.uint32))
        if ids.shape != (self.nf,):
            raise SMCError(E_ARG, "smc_batch_set_streams")
        check(lib().smc_batch_set_streams(self.ctx, ids.ctypes.data_as(_P)), "smc_batch_set_streams")

    def initialize(self):
        check(lib().smc_batch_initialize(self.ctx), "smc_batch_initialize")

    def iterate(self, n):
        check(lib().smc_batch_iterate(self.ctx, int(n)), "smc_batch_iterate")

    def run(self):
        check(lib().smc_batch_run(self.ctx), "smc_batch_run")

    def tune(self):
        """(blocks per SM, tiles per work item) chosen by the autotuner."""
        v, c = ctypes.c_int32(), ctypes.c_int32()
        check(lib().smc_batch_tune(self.ctx, ctypes.byref(v), ctypes.byref(c)), "smc_batch_tune")
        return v.value, c.value

    def log_evidence(self):
        out = np.empty(self.nf, dtype=np.float64)
        check(lib().smc_batch_log_evidence(self.ctx, out.ctypes.data_as(_P)), "smc_batch_log_evidence")
        return out

    def history(self, filter_index, count):
        recs = (Record * count)()
        n = ctypes.c_int32()
        check(lib().smc_batch_read_history(self.ctx, int(filter_index), recs, count, ctypes.byref(n)),
              "smc_batch_read_history")
        return [recs[i].as_dict() for i in range(n.value)]

    def state(self, filter_index):
        out = np.empty((4, int(self.n[filter_index])), dtype=self.rdtype)
        check(lib().smc_batch_read_state(self.ctx, int(filter_index), out.ctypes.data_as(_P), 0),
              "smc_batch_read_state")
        return out
