"""ss_sort: string sample sort with LCP output on a GB300 (sm_103a).

Thin Python binding over the C-ABI library ``_build/libss_sort.so`` (declared
in ``include/ss_sort.h``).  It only marshals arguments: every step of the sort
runs in the library's CUDA kernels.  PyTorch is used for device memory and
streams.  If the library has not been built, every call raises: there is no
fallback.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "csrc")
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD, "libss_sort.so")
ROOT = os.path.dirname(_HERE)
HEADER = os.path.join(ROOT, "include", "ss_sort.h")

SOURCES = ["ss_host.cu", "ss_big.cu", "ss_queue.cu", "ss_small.cu", "ss_merge.cu", "ss_sa.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                     "-Xcompiler", "-Wall"]

STATUS = {0: "SS_OK", 1: "SS_ERR_INVALID", 2: "SS_ERR_OOM", 3: "SS_ERR_CUDA", 4: "SS_ERR_TOO_LARGE",
          5: "SS_ERR_TIMEOUT", 6: "SS_ERR_QUEUE_FULL", 7: "SS_ERR_NO_DEVICE"}


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile every CUDA translation unit for sm_103a (in parallel) and link
    the shared library in-tree.  Returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    headers = [os.path.join(_CSRC, f) for f in os.listdir(_CSRC) if f.endswith((".cuh", ".h"))] + [HEADER]
    objs = []
    jobs = []
    for src in SOURCES:
        sp = os.path.join(_CSRC, src)
        obj = os.path.join(_BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [sp] + headers):
            jobs.append([_nvcc(), *NVCC_FLAGS, *extra_flags, "-c", sp, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    if jobs:
        with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            list(ex.map(run, jobs))
    if force or jobs or _stale(LIB_PATH, objs):
        tmp = LIB_PATH + ".tmp"
        run([_nvcc(), *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


# ---- ctypes plumbing -----------------------------------------------------------------------

class Options(ctypes.Structure):
    """Mirror of ss_options (include/ss_sort.h)."""
    _fields_ = [
        ("max_len", ctypes.c_uint32),
        ("splitters_log2", ctypes.c_uint32),
        ("big_splitters_log2", ctypes.c_uint32),
        ("tile_rounds", ctypes.c_uint32),
        ("small_cutoff", ctypes.c_uint32),
        ("big_threshold", ctypes.c_uint32),
        ("seed", ctypes.c_uint32),
        ("classifier", ctypes.c_uint32),
        ("host_parts", ctypes.c_uint32),
        ("wait_limit_us", ctypes.c_uint32),
        ("workspace", ctypes.c_void_p),
        ("workspace_bytes", ctypes.c_size_t),
    ]


class SetDesc(ctypes.Structure):
    """Mirror of ss_set."""
    _fields_ = [
        ("chars", ctypes.c_void_p),
        ("offsets", ctypes.c_void_p),
        ("n", ctypes.c_uint32),
        ("max_len", ctypes.c_uint32),
        ("out_perm", ctypes.c_void_p),
        ("out_lcp", ctypes.c_void_p),
    ]


class RunDesc(ctypes.Structure):
    """Mirror of ss_run."""
    _fields_ = [
        ("perm", ctypes.c_void_p),
        ("lcp", ctypes.c_void_p),
        ("n", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
    ]


MERGE_MAX_RUNS = 64

_lib = None


class SortError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {STATUS.get(code, code)}")


def load(path: str | None = None):
    """Load the library.  Raises if it has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"ss_sort CUDA library not built ({p}); run paper_1808_00963_gb300.build()")
    lib = ctypes.CDLL(p)
    vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    lib.ss_sort.argtypes = [vp, vp, u64, vp, vp, vp]
    lib.ss_sort.restype = i32
    lib.ss_sort_ex.argtypes = [vp, vp, u64, vp, vp, ctypes.POINTER(Options), vp]
    lib.ss_sort_ex.restype = i32
    lib.ss_workspace_size.argtypes = [u64, ctypes.POINTER(Options)]
    lib.ss_workspace_size.restype = ctypes.c_size_t
    lib.ss_sort_host.argtypes = [vp, u64, vp, u64, vp, vp, ctypes.POINTER(Options), vp]
    lib.ss_sort_host.restype = i32
    lib.ss_batch_create.argtypes = [ctypes.POINTER(SetDesc), u32, ctypes.POINTER(Options), ctypes.POINTER(vp)]
    lib.ss_batch_create.restype = i32
    lib.ss_batch_workspace_size.argtypes = [ctypes.POINTER(SetDesc), u32, ctypes.POINTER(Options)]
    lib.ss_batch_workspace_size.restype = ctypes.c_size_t
    lib.ss_batch_run.argtypes = [vp, vp]
    lib.ss_batch_run.restype = i32
    lib.ss_batch_status.argtypes = [vp, vp]
    lib.ss_batch_status.restype = i32
    lib.ss_batch_destroy.argtypes = [vp]
    lib.ss_batch_destroy.restype = i32
    lib.ss_sort_batch.argtypes = [ctypes.POINTER(SetDesc), u32, ctypes.POINTER(Options), vp]
    lib.ss_sort_batch.restype = i32
    lib.ss_status_string.argtypes = [i32]
    lib.ss_status_string.restype = ctypes.c_char_p
    lib.ss_launch_count.argtypes = []
    lib.ss_launch_count.restype = u64
    lib.ss_set_profiling.argtypes = [i32]
    lib.ss_set_profiling.restype = None
    lib.ss_set_graph_loop.argtypes = [i32]
    lib.ss_set_graph_loop.restype = None
    lib.ss_kernel_stats.argtypes = [ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(u64),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(u64), u32]
    lib.ss_kernel_stats.restype = u32
    lib.ss_reset_kernel_stats.argtypes = []
    lib.ss_reset_kernel_stats.restype = None
    lib.ss_distinguishing.argtypes = [vp, vp, u64, u32, vp, vp, vp, vp, vp, vp]
    lib.ss_distinguishing.restype = i32
    lib.ss_stream_status.argtypes = [vp]
    lib.ss_stream_status.restype = i32
    lib.ss_sort_noalloc.argtypes = [vp, vp, u64, u32, vp, vp, vp]
    lib.ss_sort_noalloc.restype = i32
    lib.ss_merge.argtypes = [vp, vp, u32, ctypes.POINTER(RunDesc), u32, u32, vp, vp, vp, ctypes.c_size_t, vp]
    lib.ss_merge.restype = i32
    lib.ss_merge_workspace_size.argtypes = [ctypes.POINTER(RunDesc), u32, u32]
    lib.ss_merge_workspace_size.restype = ctypes.c_size_t
    lib.ss_sort_dna.argtypes = [vp, u64, vp, u64, vp, vp, ctypes.POINTER(Options), vp]
    lib.ss_sort_dna.restype = i32
    lib.ss_suffix_array.argtypes = [vp, u64, vp, vp, u32, vp]
    lib.ss_suffix_array.restype = i32
    if path is None:
        _lib = lib
    return lib


def make_options(max_len=0, **kw) -> Options:
    o = Options()
    o.max_len = max_len
    for k, v in kw.items():
        if v is not None:
            setattr(o, k, v)
    return o


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(code, what):
    if code != 0:
        raise SortError(code, what)


def sort(chars, offsets, max_len: int = 0, with_lcp: bool = True, out=None, stream=None, dna: bool = False,
         sync: bool = True, **opts):
    """Sort the strings of a device string set.

    chars   : torch.uint8 CUDA tensor (NUL-terminated strings)
    offsets : torch.int64 CUDA tensor (start of each string)
    dna     : the bytes of chars are only A, C, G, T and terminators: sort
              with 3-bit character codes, 21 characters per key
    sync    : wait for the sort and raise SortError on a device-side error
              (ss_stream_status); False only enqueues it (ss_sort_ex is
              asynchronous), and the caller reads the status later with
              stream_status()
    Returns (perm, lcp) as torch.int32 CUDA tensors holding uint32 values
    (lcp is None when with_lcp is False), on the current stream (or
    ``stream``).
    """
    import torch
    lib = load()
    n = int(offsets.numel())
    dev = offsets.device
    if out is None:
        perm = torch.empty(n, dtype=torch.int32, device=dev)
        lcp = torch.empty(n, dtype=torch.int32, device=dev) if with_lcp else None
    else:
        perm, lcp = out
    assert chars.dtype == torch.uint8 and chars.is_cuda and chars.is_contiguous()
    assert offsets.dtype == torch.int64 and offsets.is_cuda and offsets.is_contiguous()
    o = make_options(max_len, **opts)
    lp = ctypes.c_void_p(lcp.data_ptr()) if lcp is not None else None
    if dna:
        rc = lib.ss_sort_dna(ctypes.c_void_p(chars.data_ptr()), int(chars.numel()),
                             ctypes.c_void_p(offsets.data_ptr()), n, ctypes.c_void_p(perm.data_ptr()), lp,
                             ctypes.byref(o), _stream_ptr(stream))
        _check(rc, "ss_sort_dna")
    else:
        rc = lib.ss_sort_ex(ctypes.c_void_p(chars.data_ptr()), ctypes.c_void_p(offsets.data_ptr()), n,
                            ctypes.c_void_p(perm.data_ptr()), lp, ctypes.byref(o), _stream_ptr(stream))
        _check(rc, "ss_sort_ex")
        if sync:
            _check(lib.ss_stream_status(_stream_ptr(stream)), "ss_sort_ex (device status)")
    return perm, lcp


def stream_status(stream=None):
    """ss_stream_status: wait for the stream and raise SortError if a sort
    enqueued on it latched a device-side error."""
    _check(load().ss_stream_status(_stream_ptr(stream)), "ss_stream_status")


def distinguishing(chars, offsets, perm, lcp, max_len: int = 0, stream=None):
    """Distinguishing character c^_j (uint8) and distinguishing-prefix length
    d_j (int32) of every sorted position, and D = sum d_j (Section 4.3.4,
    Lemma 2.1), from the outputs of sort()."""
    import torch
    lib = load()
    n = int(perm.numel())
    dchar = torch.empty(n, dtype=torch.uint8, device=perm.device)
    dpre = torch.empty(n, dtype=torch.int32, device=perm.device)
    D = torch.zeros(1, dtype=torch.int64, device=perm.device)
    rc = lib.ss_distinguishing(ctypes.c_void_p(chars.data_ptr()), ctypes.c_void_p(offsets.data_ptr()), n, max_len,
                               ctypes.c_void_p(perm.data_ptr()), ctypes.c_void_p(lcp.data_ptr()),
                               ctypes.c_void_p(dchar.data_ptr()), ctypes.c_void_p(dpre.data_ptr()),
                               ctypes.c_void_p(D.data_ptr()), _stream_ptr(stream))
    _check(rc, "ss_distinguishing")
    return dchar, dpre, D


def _run_descs(runs):
    arr = (RunDesc * max(1, len(runs)))()
    for k, (perm, lcp) in enumerate(runs):
        n = int(perm.numel())
        if int(lcp.numel()) != n:
            raise ValueError("each run needs one LCP entry per string")
        arr[k].perm = perm.data_ptr() if n else None
        arr[k].lcp = lcp.data_ptr() if n else None
        arr[k].n = n
        arr[k].reserved = 0
    return arr


def merge_workspace_size(runs, sample_step: int = 0) -> int:
    """Device workspace bytes merge() needs for these runs."""
    return int(load().ss_merge_workspace_size(_run_descs(runs), len(runs), sample_step))


def merge(chars, offsets, runs, max_len: int = 0, with_lcp: bool = True, out=None, sample_step: int = 0,
          workspace=None, workspace_bytes: int = 0, stream=None):
    """Merge sorted runs (a list of (perm, lcp) int32 device tensors holding
    indices into the string set (chars, offsets), each sorted as sort() sorts)
    into one sorted order and its LCP array (Section 4.3.2, Algorithm 4.5).
    Asynchronous on ``stream``."""
    import torch
    lib = load()
    total = sum(int(r[0].numel()) for r in runs)
    dev = runs[0][0].device if runs else chars.device
    if out is None:
        perm = torch.empty(total, dtype=torch.int32, device=dev)
        lcp = torch.empty(total, dtype=torch.int32, device=dev) if with_lcp else None
    else:
        perm, lcp = out
    rc = lib.ss_merge(ctypes.c_void_p(chars.data_ptr()), ctypes.c_void_p(offsets.data_ptr()), max_len,
                      _run_descs(runs), len(runs), sample_step, ctypes.c_void_p(perm.data_ptr()),
                      ctypes.c_void_p(lcp.data_ptr()) if lcp is not None else None,
                      ctypes.c_void_p(workspace) if workspace else None, workspace_bytes, _stream_ptr(stream))
    _check(rc, "ss_merge")
    return perm, lcp


def suffix_array(text, n: int | None = None, with_lcp: bool = True, initial_depth: int = 0, out=None,
                 stream=None):
    """Suffix array (int32) and LCP array of a text held on the device as n
    bytes in 1..255 followed by a zero byte (Section 8.2, prefix doubling on
    top of the string sort)."""
    import torch
    lib = load()
    if n is None:
        n = int(text.numel()) - 1
    if out is None:
        sa = torch.empty(n, dtype=torch.int32, device=text.device)
        lcp = torch.empty(n, dtype=torch.int32, device=text.device) if with_lcp else None
    else:
        sa, lcp = out
    rc = lib.ss_suffix_array(ctypes.c_void_p(text.data_ptr()), n, ctypes.c_void_p(sa.data_ptr()),
                             ctypes.c_void_p(lcp.data_ptr()) if lcp is not None else None, initial_depth,
                             _stream_ptr(stream))
    _check(rc, "ss_suffix_array")
    return sa, lcp


def sort_host(chars, offsets, max_len: int = 0, with_lcp: bool = True, perm=None, lcp=None, stream=None,
              **opts):
    """Sort a host string set (numpy arrays or CPU tensors, ideally pinned):
    the copies to and from the device happen inside the library call.
    host_parts=P (a power of two <= 16) sorts P parts while later ones are
    still being copied and LCP-merges them (strings packed in index order;
    other layouts are sorted again in one piece)."""
    import numpy as np
    lib = load()

    def ptr(a):
        return ctypes.c_void_p(a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data)

    n = int(offsets.shape[0])
    if perm is None:
        perm = np.empty(n, np.uint32)
    if with_lcp and lcp is None:
        lcp = np.empty(n, np.uint32)
    o = make_options(max_len, **opts)
    nbytes = int(chars.numel() if hasattr(chars, "numel") else chars.size)
    rc = lib.ss_sort_host(ptr(chars), nbytes, ptr(offsets), n, ptr(perm), ptr(lcp) if with_lcp else None,
                          ctypes.byref(o), _stream_ptr(stream))
    _check(rc, "ss_sort_host")
    return perm, (lcp if with_lcp else None)


NOALLOC_MAX_STRINGS = 65536


def sort_noalloc(chars, offsets, max_len: int = 0, out=None, stream=None):
    """ss_sort_noalloc: sort up to 65536 strings without any allocation by the
    library (its workspace is a fixed array in the library's device data).
    ``out`` = (perm, lcp) preallocated int32 CUDA tensors (lcp may be None);
    callers that may not allocate pass their own.  Returns (perm, lcp)."""
    import torch
    lib = load()
    n = int(offsets.numel())
    if out is None:
        out = (torch.empty(n, dtype=torch.int32, device=offsets.device),
               torch.empty(n, dtype=torch.int32, device=offsets.device))
    perm, lcp = out
    rc = lib.ss_sort_noalloc(ctypes.c_void_p(chars.data_ptr()), ctypes.c_void_p(offsets.data_ptr()), n, max_len,
                             ctypes.c_void_p(perm.data_ptr()),
                             ctypes.c_void_p(lcp.data_ptr()) if lcp is not None else None, _stream_ptr(stream))
    _check(rc, "ss_sort_noalloc")
    return perm, lcp


def workspace_size(n: int, max_len: int = 0, **opts) -> int:
    o = make_options(max_len, **opts)
    return int(load().ss_workspace_size(n, ctypes.byref(o)))


class Batch:
    """A planned batch of independent string sets (ss_batch_create / _run).

    sets: list of (chars, offsets, max_len, perm_out, lcp_out) with CUDA
    tensors (lcp_out may be None).  ``run()`` only enqueues work, so it can be
    captured into a CUDA graph; ``status()`` waits and reports errors.
    """

    def __init__(self, sets, own_workspace: bool = False, **opts):
        self.lib = load()
        self.keep = sets
        arr = (SetDesc * max(1, len(sets)))()
        for i, (ch, off, ml, p, l) in enumerate(sets):
            arr[i].chars = ch.data_ptr()
            arr[i].offsets = off.data_ptr()
            arr[i].n = int(off.numel())
            arr[i].max_len = int(ml)
            arr[i].out_perm = p.data_ptr()
            arr[i].out_lcp = l.data_ptr() if l is not None else None
        self.arr = arr
        self.opts = make_options(0, **opts)
        self.work = None
        if own_workspace:
            # workspace from the caller's (torch's) allocator instead of the library's
            import torch
            nb = int(self.lib.ss_batch_workspace_size(arr, len(sets), ctypes.byref(self.opts)))
            self.work = torch.empty(max(nb, 256), dtype=torch.uint8, device="cuda")
            self.opts.workspace = self.work.data_ptr()
            self.opts.workspace_bytes = nb
        h = ctypes.c_void_p()
        _check(self.lib.ss_batch_create(arr, len(sets), ctypes.byref(self.opts), ctypes.byref(h)),
               "ss_batch_create")
        self.h = h

    def run(self, stream=None):
        _check(self.lib.ss_batch_run(self.h, _stream_ptr(stream)), "ss_batch_run")

    def status(self, stream=None):
        _check(self.lib.ss_batch_status(self.h, _stream_ptr(stream)), "ss_batch_status")

    def stream_status(self, stream=None):
        """ss_stream_status on the stream this batch last ran on."""
        _check(self.lib.ss_stream_status(_stream_ptr(stream)), "ss_stream_status")

    def close(self):
        if self.h:
            self.lib.ss_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count() -> int:
    return int(load().ss_launch_count())


def set_profiling(on: bool):
    load().ss_set_profiling(1 if on else 0)


def set_graph_loop(on: bool):
    """ss_set_graph_loop: run the multi-block rounds as one graph launch
    (default) or launch by launch from the host (for kernel profilers)."""
    load().ss_set_graph_loop(1 if on else 0)


def reset_kernel_stats():
    load().ss_reset_kernel_stats()


def kernel_stats():
    """{kernel class: (launches, total_ms, algorithmic_bytes)} recorded while
    profiling was on."""
    lib = load()
    cap = 64
    names = (ctypes.c_char_p * cap)()
    la = (ctypes.c_uint64 * cap)()
    ms = (ctypes.c_double * cap)()
    by = (ctypes.c_uint64 * cap)()
    k = lib.ss_kernel_stats(names, la, ms, by, cap)
    return {names[i].decode(): (int(la[i]), float(ms[i]), int(by[i])) for i in range(min(k, cap))}
