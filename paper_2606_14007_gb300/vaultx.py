"""Python binding of the VaultxGPU C ABI (include/vaultx.h), via ctypes.

Argument marshalling only: every step of the plotting path runs in the CUDA
kernels of ``libvaultx.so``.  PyTorch supplies device memory (``torch.empty``
on ``cuda``) and streams.  There is no CPU fallback: if the library is not
built, :func:`lib` raises.

Functions keep the C names (``vx_plot_create``, ``vx_table1``, ``vx_match``,
``vx_plot_batch``, ``vx_serve_submit`` ...).  :class:`Plot` is a small
convenience owner of one plot and its torch buffers.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libvaultx.so")

VX_OK, VX_EINVAL, VX_ENOMEM, VX_ECUDA, VX_ETIMEDOUT, VX_EBUSY, VX_ENOTREADY, VX_EOVERFLOW, VX_EIO = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
VX_TABLE1, VX_TABLE2 = 1, 2
VX_TEST_WITHHOLD_PREFIX = 1
VX_QUEUED, VX_RUNNING, VX_DONE, VX_FAILED = 0, 1, 2, 3
T1_REC, T2_REC = 12, 16


class VxError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str = ""):
        self.code = code
        msg = "%s failed: %s (%d)" % (what, strerror(code) if _lib else "", code)
        if detail:
            msg += ": " + detail
        super().__init__(msg)


class vx_opts(ctypes.Structure):
    _fields_ = [
        ("size", ctypes.c_uint32),
        ("test_flags", ctypes.c_uint32),
        ("match_distance", ctypes.c_uint64),
        ("partition_log2", ctypes.c_int32),
        ("coarse_bits", ctypes.c_int32),
        ("slack_sigma", ctypes.c_uint32),
        ("hash_block", ctypes.c_uint32),
        ("nonces_per_thread", ctypes.c_uint32),
        ("scatter_mode", ctypes.c_uint32),
        ("t2_capacity", ctypes.c_uint64),
        ("fuse_pair_hash", ctypes.c_uint32),
        ("pipeline_chunks", ctypes.c_uint32),
        ("t2_placement", ctypes.c_uint32),
        ("match_scope", ctypes.c_uint32),
        ("window_bits", ctypes.c_uint32),
        ("window", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32 * 2),
    ]


class vx_serve_opts(ctypes.Structure):
    _fields_ = [
        ("size", ctypes.c_uint32),
        ("max_inflight", ctypes.c_uint32),
        ("memory_budget", ctypes.c_uint64),
        ("streams", ctypes.c_uint32),
        ("max_wave", ctypes.c_uint32),
        ("plot_opts", vx_opts),
    ]


_lib = None
_lock = threading.Lock()


def lib():
    """The loaded libvaultx.so.  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError("libvaultx.so is not built (run __graft_entry__.build() or "
                              "python -m paper_2606_14007_gb300._build); no CPU fallback exists")
        L = ctypes.CDLL(LIB_PATH)
        vp, c_int, u64, u32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32
        u8p = ctypes.c_char_p
        P = ctypes.POINTER
        sig = {
            "vx_version": (c_int, []),
            "vx_opts_default": (c_int, [P(vx_opts)]),
            "vx_strerror": (ctypes.c_char_p, [c_int]),
            "vx_last_error": (ctypes.c_char_p, [vp]),
            "vx_plot_required_bytes": (c_int, [c_int, P(vx_opts), P(u64), P(u64), P(u64)]),
            "vx_plot_create": (c_int, [c_int, u8p, P(vx_opts), P(vp)]),
            "vx_plot_bind": (c_int, [vp, vp, vp, vp, u64]),
            "vx_plot_alloc": (c_int, [vp]),
            "vx_table1": (c_int, [vp, vp]),
            "vx_match": (c_int, [vp, vp]),
            "vx_plot_run": (c_int, [vp, vp]),
            "vx_sync": (c_int, [vp]),
            "vx_table_info": (c_int, [vp, c_int, P(vp), P(u64), P(u32)]),
            "vx_table1_offsets": (c_int, [vp, vp, vp]),
            "vx_table_copy": (c_int, [vp, c_int, u64, vp, u64, vp]),
            "vx_plot_write": (c_int, [vp, ctypes.c_char_p, P(ctypes.c_double), P(ctypes.c_double)]),
            "vx_sort_table2_work_bytes": (c_int, [vp, P(u64)]),
            "vx_autotune": (c_int, [c_int, P(vx_opts), P(vx_opts), P(ctypes.c_double), vp]),
            "vx_sort_table2": (c_int, [vp, vp, u64, vp]),
            "vx_plot_batch": (c_int, [P(vp), c_int, vp]),
            "vx_plot_tiled_bytes": (c_int, [c_int, P(vx_opts), c_int, P(u64), P(u64), P(u64)]),
            "vx_plot_tiled_window_bits": (c_int, [c_int, P(vx_opts), u64, P(c_int)]),
            "vx_plot_tiled_window_bits_capped": (c_int, [c_int, P(vx_opts), u64, u32, P(c_int)]),
            "vx_plot_tiled_hash_passes": (c_int, [c_int, P(vx_opts), c_int, P(u32)]),
            "vx_plot_tiled": (c_int, [c_int, u8p, P(vx_opts), c_int, vp, u64, vp, u64, vp, u64, P(u64),
                                      P(u64), vp]),
            "vx_plot_tiled_write": (c_int, [c_int, u8p, P(vx_opts), c_int, vp, u64, ctypes.c_char_p, vp,
                                            u64, P(u64), P(u64), P(ctypes.c_double), vp]),
            "vx_plot_destroy": (None, [vp]),
            "vx_plot_run_noalloc": (c_int, [c_int, u8p, P(vx_opts), vp, vp, u64, vp, P(u64)]),
            "vx_hash_nonces": (c_int, [u8p, u64, u64, vp, vp]),
            "vx_pair_hash": (c_int, [u8p, vp, u64, vp, vp]),
            "vx_hash_peak": (c_int, [u8p, u64, u64, vp, u32, vp]),
            "vx_test_fail_next_allocs": (c_int, [c_int]),
            "vx_plot_profile": (c_int, [vp, c_int]),
            "vx_plot_profile_read": (c_int, [vp, P(ctypes.c_double), c_int, P(c_int), P(c_int)]),
            "vx_kernel_name": (ctypes.c_char_p, [c_int]),
            "vx_plot_kernel_mask": (c_int, [vp, c_int, P(u32)]),
            "vx_serve_create": (c_int, [P(vx_serve_opts), P(vp)]),
            "vx_serve_submit": (c_int, [vp, c_int, u8p, P(u64)]),
            "vx_serve_poll": (c_int, [vp, u64, P(c_int), P(vp)]),
            "vx_serve_step": (c_int, [vp]),
            "vx_serve_latency": (c_int, [vp, u64, P(ctypes.c_double)]),
            "vx_serve_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def strerror(code: int) -> str:
    return lib().vx_strerror(code).decode()


def last_error(plot) -> str:
    return lib().vx_last_error(plot).decode()


def _check(rc: int, what: str, plot=None):
    if rc != VX_OK:
        detail = lib().vx_last_error(plot).decode() if plot else ""
        raise VxError(rc, what, detail)
    return rc


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _key(key: bytes) -> bytes:
    key = bytes(key)
    if len(key) != 32:
        raise ValueError("plot key must be 32 bytes")
    return key


# ------------------------------------------------------------ C names --

def vx_opts_default() -> vx_opts:
    o = vx_opts()
    _check(lib().vx_opts_default(ctypes.byref(o)), "vx_opts_default")
    return o


def make_opts(**kw) -> vx_opts:
    o = vx_opts_default()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def vx_plot_required_bytes(K: int, opts: vx_opts | None = None) -> tuple[int, int, int]:
    a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().vx_plot_required_bytes(K, ctypes.byref(opts) if opts else None, ctypes.byref(a),
                                        ctypes.byref(b), ctypes.byref(c)), "vx_plot_required_bytes")
    return a.value, b.value, c.value


def vx_plot_create(K: int, key: bytes, opts: vx_opts | None = None) -> int:
    h = ctypes.c_void_p()
    _check(lib().vx_plot_create(K, _key(key), ctypes.byref(opts) if opts else None,
                                ctypes.byref(h)), "vx_plot_create")
    return h.value


def vx_plot_bind(plot, d_t1: int, d_t2: int, d_scratch: int, t2_capacity: int = 0):
    return _check(lib().vx_plot_bind(plot, d_t1, d_t2, d_scratch, t2_capacity), "vx_plot_bind", plot)


def vx_plot_alloc(plot):
    return _check(lib().vx_plot_alloc(plot), "vx_plot_alloc", plot)


def vx_table1(plot, stream=None):
    return _check(lib().vx_table1(plot, _stream(stream)), "vx_table1", plot)


def vx_match(plot, stream=None):
    return _check(lib().vx_match(plot, _stream(stream)), "vx_match", plot)


def vx_plot_run(plot, stream=None):
    return _check(lib().vx_plot_run(plot, _stream(stream)), "vx_plot_run", plot)


def vx_sync(plot, check: bool = True) -> int:
    rc = lib().vx_sync(plot)
    return _check(rc, "vx_sync", plot) if check else rc


def vx_table_info(plot, which: int, check: bool = True):
    p, n, rb = ctypes.c_void_p(), ctypes.c_uint64(), ctypes.c_uint32()
    rc = lib().vx_table_info(plot, which, ctypes.byref(p), ctypes.byref(n), ctypes.byref(rb))
    if check:
        _check(rc, "vx_table_info", plot)
    return (p.value or 0), n.value, rb.value, rc


def vx_table1_offsets(plot, d_out: int, stream=None):
    return _check(lib().vx_table1_offsets(plot, d_out, _stream(stream)), "vx_table1_offsets", plot)


def vx_table_copy(plot, which: int, host_dst: int, nbytes: int, stream=None, offset: int = 0):
    return _check(lib().vx_table_copy(plot, which, offset, host_dst, nbytes, _stream(stream)),
                  "vx_table_copy", plot)


def vx_autotune(K: int, opts: vx_opts | None = None, stream=None) -> tuple[vx_opts, float]:
    """The fastest plan for K on this device (library timing, no cache)."""
    best, ms = vx_opts(), ctypes.c_double()
    _check(lib().vx_autotune(K, ctypes.byref(opts) if opts else None, ctypes.byref(best),
                             ctypes.byref(ms), _stream(stream)), "vx_autotune")
    return best, ms.value


_TUNED = ("partition_log2", "scatter_mode", "nonces_per_thread")


def autotune(K: int, opts: vx_opts | None = None, cache_path: str | None = None,
             stream=None) -> vx_opts:
    """vx_autotune with an on-disk cache keyed by (device, K, base options):
    the first call times the candidates, later calls (any process) reuse the
    choice.  Cache file: cache_path, else $VX_TUNE_CACHE, else
    ~/.cache/vaultx/tune.json."""
    import json
    import os
    import torch
    path = cache_path or os.environ.get("VX_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "vaultx", "tune.json")
    base = opts if opts is not None else vx_opts_default()
    prop = torch.cuda.get_device_properties(torch.cuda.current_device())
    fields = {n: getattr(base, n) for n, _ in vx_opts._fields_
              if n not in ("size", "reserved") + _TUNED}
    key = json.dumps([prop.name, prop.multi_processor_count, K, fields], sort_keys=True)
    try:
        with open(path) as f:
            cache = json.load(f)
    except (OSError, ValueError):
        cache = {}
    out = vx_opts()
    ctypes.memmove(ctypes.byref(out), ctypes.byref(base), ctypes.sizeof(vx_opts))
    if key in cache:
        for n in _TUNED:
            setattr(out, n, int(cache[key].get(n, 0)))
        return out
    best, ms = vx_autotune(K, base, stream)
    entry = {n: int(getattr(best, n)) for n in _TUNED}
    entry["ms"] = ms
    cache[key] = entry
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, path)
    for n in _TUNED:
        setattr(out, n, entry[n])
    return out


def vx_sort_table2_work_bytes(plot) -> int:
    n = ctypes.c_uint64()
    _check(lib().vx_sort_table2_work_bytes(plot, ctypes.byref(n)), "vx_sort_table2_work_bytes", plot)
    return n.value


def vx_sort_table2(plot, d_work: int, work_bytes: int, stream=None):
    """Table 2 reordered in place by (key2, a, b), key2 = big-endian hash2;
    asynchronous, vx_sync reports its status."""
    return _check(lib().vx_sort_table2(plot, d_work, work_bytes, _stream(stream)), "vx_sort_table2",
                  plot)


def vx_plot_write(plot, path: str) -> tuple[float, float]:
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().vx_plot_write(plot, path.encode(), ctypes.byref(a), ctypes.byref(b)),
           "vx_plot_write", plot)
    return a.value, b.value


def vx_plot_batch(plots, stream=None):
    arr = (ctypes.c_void_p * len(plots))(*plots)
    rc = lib().vx_plot_batch(arr, len(plots), _stream(stream))
    return _check(rc, "vx_plot_batch", plots[0] if plots else None)


def vx_plot_destroy(plot):
    if plot:
        lib().vx_plot_destroy(plot)


def vx_plot_tiled_bytes(K: int, window_bits: int, opts: vx_opts | None = None) -> tuple[int, int, int]:
    """(device bytes, host Table-1 bytes, host Table-2 bound) of a tiled plot."""
    a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().vx_plot_tiled_bytes(K, ctypes.byref(opts) if opts else None, window_bits,
                                     ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "vx_plot_tiled_bytes")
    return a.value, b.value, c.value


def vx_plot_tiled_window_bits(K: int, budget_bytes: int, opts: vx_opts | None = None,
                              max_hash_passes: int | None = None) -> int:
    """The fewest window bits whose tiled device footprint fits budget_bytes
    (with at most max_hash_passes hashes of every nonce; default 2, the
    window-id path)."""
    c = ctypes.c_int()
    o = ctypes.byref(opts) if opts else None
    if max_hash_passes is None:
        _check(lib().vx_plot_tiled_window_bits(K, o, budget_bytes, ctypes.byref(c)),
               "vx_plot_tiled_window_bits")
    else:
        _check(lib().vx_plot_tiled_window_bits_capped(K, o, budget_bytes, max_hash_passes, ctypes.byref(c)),
               "vx_plot_tiled_window_bits_capped")
    return c.value


def vx_plot_tiled_hash_passes(K: int, window_bits: int, opts: vx_opts | None = None) -> int:
    """How many times a tiled plot hashes every nonce at window_bits."""
    n = ctypes.c_uint32()
    _check(lib().vx_plot_tiled_hash_passes(K, ctypes.byref(opts) if opts else None, window_bits,
                                           ctypes.byref(n)), "vx_plot_tiled_hash_passes")
    return n.value


def vx_plot_tiled(K: int, key: bytes, window_bits: int, host_t1: int, host_t1_bytes: int,
                  host_t2: int, host_t2_bytes: int, opts: vx_opts | None = None, stream=None,
                  check: bool = True, d_work: int = 0, work_bytes: int = 0):
    """Whole plot one window at a time, tables copied to host memory at
    host_t1 (0 = skip Table 1) and host_t2; window buffers cut from d_work
    (device, 0 = allocated for the call); synchronous.  Returns (status,
    Table-1 records, Table-2 records)."""
    n1, n2 = ctypes.c_uint64(), ctypes.c_uint64()
    rc = lib().vx_plot_tiled(K, _key(key), ctypes.byref(opts) if opts else None, window_bits,
                             d_work or None, work_bytes, host_t1 or None, host_t1_bytes, host_t2,
                             host_t2_bytes, ctypes.byref(n1), ctypes.byref(n2), _stream(stream))
    if check:
        _check(rc, "vx_plot_tiled")
    return rc, n1.value, n2.value


def vx_plot_tiled_write(K: int, key: bytes, window_bits: int, path: str, host_t1: int = 0,
                        host_t1_bytes: int = 0, opts: vx_opts | None = None, stream=None,
                        check: bool = True, d_work: int = 0, work_bytes: int = 0):
    """Whole plot one window at a time, Table 2 written as a flat plot file
    at `path` (Table 1 copied to host_t1 unless 0); window buffers cut from
    d_work (0 = allocated for the call); synchronous.  Returns (status,
    Table-1 records, Table-2 records, seconds)."""
    n1, n2, sec = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_double()
    rc = lib().vx_plot_tiled_write(K, _key(key), ctypes.byref(opts) if opts else None, window_bits,
                                   d_work or None, work_bytes, path.encode(), host_t1 or None,
                                   host_t1_bytes, ctypes.byref(n1), ctypes.byref(n2), ctypes.byref(sec),
                                   _stream(stream))
    if check:
        _check(rc, "vx_plot_tiled_write")
    return rc, n1.value, n2.value, sec.value


def plot_tiled(K: int, key: bytes, window_bits: int | None, opts: vx_opts | None = None,
               table1: bool = True, pin: bool = True, stream=None, work=None, budget: int = 0):
    """vx_plot_tiled into fresh host tensors: returns (t1, t2), uint8 views
    shaped (records, 12) and (records, 16) (t1 None unless table1).  `work`:
    an optional uint8 device tensor of at least vx_plot_tiled_bytes' device
    bytes for the window buffers.  window_bits None: the fewest that fit
    `budget` bytes of device memory."""
    import torch
    if window_bits is None:
        window_bits = vx_plot_tiled_window_bits(K, budget, opts)
    _, h1, h2 = vx_plot_tiled_bytes(K, window_bits, opts)
    t1 = torch.empty(h1 if table1 else 0, dtype=torch.uint8, pin_memory=pin)
    t2 = torch.empty(h2, dtype=torch.uint8, pin_memory=pin)
    _, n1, n2 = vx_plot_tiled(K, key, window_bits, t1.data_ptr() if table1 else 0, h1 if table1 else 0,
                              t2.data_ptr(), h2, opts, stream,
                              d_work=work.data_ptr() if work is not None else 0,
                              work_bytes=work.numel() if work is not None else 0)
    return (t1[: T1_REC * n1].view(n1, T1_REC) if table1 else None,
            t2[: T2_REC * n2].view(n2, T2_REC))


def vx_plot_run_noalloc(K: int, key: bytes, d_t1: int, d_t2: int, t2_capacity: int = 0,
                        opts: vx_opts | None = None, stream=None, check: bool = True):
    """Whole plot with the library's static scratch array (no allocation);
    synchronous.  Returns (status, Table-2 record count)."""
    n = ctypes.c_uint64()
    rc = lib().vx_plot_run_noalloc(K, _key(key), ctypes.byref(opts) if opts else None, d_t1, d_t2,
                                   t2_capacity, _stream(stream), ctypes.byref(n))
    if check:
        _check(rc, "vx_plot_run_noalloc")
    return rc, n.value


def vx_hash_nonces(key: bytes, nonce0: int, count: int, d_out: int, stream=None):
    return _check(lib().vx_hash_nonces(_key(key), nonce0, count, d_out, _stream(stream)),
                  "vx_hash_nonces")


def vx_hash_peak(key: bytes, nonce0: int, count: int, d_fold: int, fold_words: int, stream=None):
    """Hash-only ceiling: count keyed hashes, folded per thread into d_fold."""
    return _check(lib().vx_hash_peak(_key(key), nonce0, count, d_fold, fold_words, _stream(stream)),
                  "vx_hash_peak")


def vx_pair_hash(key: bytes, d_pairs: int, count: int, d_out: int, stream=None):
    return _check(lib().vx_pair_hash(_key(key), d_pairs, count, d_out, _stream(stream)),
                  "vx_pair_hash")


def vx_plot_profile(plot, runs: int):
    return _check(lib().vx_plot_profile(plot, runs), "vx_plot_profile", plot)


def vx_plot_profile_read(plot) -> tuple[dict, int]:
    """({kernel name: total ms over the traced runs}, runs)."""
    ms = (ctypes.c_double * 16)()
    nk, nr = ctypes.c_int(), ctypes.c_int()
    _check(lib().vx_plot_profile_read(plot, ms, 16, ctypes.byref(nk), ctypes.byref(nr)),
           "vx_plot_profile_read", plot)
    return {lib().vx_kernel_name(k).decode(): ms[k] for k in range(nk.value)}, nr.value


def vx_plot_kernel_mask(plot, split: bool = False) -> list[str]:
    """Names of the kernels one run of the plot launches."""
    m = ctypes.c_uint32()
    _check(lib().vx_plot_kernel_mask(plot, 1 if split else 0, ctypes.byref(m)),
           "vx_plot_kernel_mask", plot)
    return [lib().vx_kernel_name(k).decode() for k in range(32) if m.value >> k & 1]


def vx_test_fail_next_allocs(count: int):
    return lib().vx_test_fail_next_allocs(count)


def vx_serve_create(opts: vx_serve_opts | None = None) -> int:
    h = ctypes.c_void_p()
    _check(lib().vx_serve_create(ctypes.byref(opts) if opts else None, ctypes.byref(h)),
           "vx_serve_create")
    return h.value


def vx_serve_submit(srv, K: int, key: bytes) -> int:
    t = ctypes.c_uint64()
    _check(lib().vx_serve_submit(srv, K, _key(key), ctypes.byref(t)), "vx_serve_submit")
    return t.value


def vx_serve_poll(srv, ticket: int, take: bool = True):
    st, h = ctypes.c_int(), ctypes.c_void_p()
    _check(lib().vx_serve_poll(srv, ticket, ctypes.byref(st), ctypes.byref(h) if take else None),
           "vx_serve_poll")
    return st.value, h.value


def vx_serve_step(srv) -> int:
    rc = lib().vx_serve_step(srv)
    if rc < 0:
        raise VxError(rc, "vx_serve_step")
    return rc


def vx_serve_latency(srv, ticket: int) -> float:
    s = ctypes.c_double()
    _check(lib().vx_serve_latency(srv, ticket, ctypes.byref(s)), "vx_serve_latency")
    return s.value


def vx_serve_destroy(srv):
    if srv:
        lib().vx_serve_destroy(srv)


# --------------------------------------------------------- convenience --

class Plot:
    """One plot with torch-allocated device buffers bound to it.

    ``Plot(K, key).run()`` issues the fused plot (``run_split()``: vx_table1
    + vx_match) on the current torch stream; ``sync()`` waits and returns the
    Table-2 count; ``t1`` / ``t2`` are zero-copy uint8 views shaped
    (records, 12) / (records, 16).  With ``vx_opts.window_bits`` the plot is
    one window of the whole plot, and ``t1`` holds the window's records
    (their count is known after ``sync()``).
    """

    def __init__(self, K: int, key: bytes, opts: vx_opts | None = None, device=None):
        import torch
        self.K, self.key = K, _key(key)
        self.opts = opts
        self.handle = vx_plot_create(K, key, opts)
        t1b, t2b, sb = vx_plot_required_bytes(K, opts)
        dev = torch.device("cuda") if device is None else torch.device(device)
        self._t1 = torch.empty(t1b, dtype=torch.uint8, device=dev)
        self._t2 = torch.empty(t2b, dtype=torch.uint8, device=dev)
        self._scratch = torch.empty(sb, dtype=torch.uint8, device=dev)
        self.t2_capacity = (t2b - 256) // T2_REC
        vx_plot_bind(self.handle, self._t1.data_ptr(), self._t2.data_ptr(),
                     self._scratch.data_ptr(), 0)
        self.n1 = 1 << K
        self.n2 = None

    def table1(self, stream=None):
        vx_table1(self.handle, stream)
        return self

    def match(self, stream=None):
        vx_match(self.handle, stream)
        return self

    def run(self, stream=None):
        """Both tables in one pass (fused sort + match)."""
        vx_plot_run(self.handle, stream)
        return self

    def run_split(self, stream=None):
        """Both tables through vx_table1 then vx_match."""
        return self.table1(stream).match(stream)

    def sync(self) -> int:
        vx_sync(self.handle)
        _, n, _, _ = vx_table_info(self.handle, VX_TABLE2, check=False)
        self.n2 = n
        _, n1, _, _ = vx_table_info(self.handle, VX_TABLE1, check=False)
        self.n1 = n1  # a window's share of the 2^K records
        return n

    @property
    def t1(self):
        return self._t1[: T1_REC * self.n1].view(self.n1, T1_REC)

    @property
    def t2(self):
        if self.n2 is None:
            raise RuntimeError("call sync() after match() first")
        return self._t2[: T2_REC * self.n2].view(self.n2, T2_REC)

    def offsets(self, stream=None):
        import torch
        out = torch.empty((1 << 24) + 1, dtype=torch.int64, device=self._t1.device)
        vx_table1_offsets(self.handle, out.data_ptr(), stream)
        return out

    def close(self):
        if self.handle:
            vx_plot_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
