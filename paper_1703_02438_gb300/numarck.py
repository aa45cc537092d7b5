"""Thin Python binding of libnumarck.so (the C ABI of include/numarck.h).

Argument marshalling only: every step of compression and decompression runs in the library's
CUDA kernels. torch supplies device memory and the current CUDA stream. If the library has not
been built, every call raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import struct

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libnumarck.so")

OK = 0
ERR_INVALID_ARG = 1
ERR_CAPACITY = 2
ERR_CUDA = 3
ERR_CORRUPT = 4
ERR_RANGE = 5
ERR_TIMEOUT = 6
ERR_NOMEM = 7
F32 = 0
F64 = 1
ANCHOR_ZERO = 0
ANCHOR_MIN = 1
HEADER_BYTES = 256

HEADER_FIELDS = ("magic", "version", "dtype", "B", "E", "anchor", "status", "n", "block_bytes",
                 "epb", "nblocks", "sub", "nsub", "n_sel", "n_inc", "a", "block_stride",
                 "off_centres", "off_idx_off", "off_inc_off", "off_sub_off", "off_index",
                 "off_exact", "total_bytes")
_HEADER_FMT = "<IIiidiiqqqqqqqqdqqqqqqqq"


class NumarckError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} (status {code})")


class Params(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("B", ctypes.c_int32), ("E", ctypes.c_double),
                ("anchor", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("block_bytes", ctypes.c_int64)]


class BatchItem(ctypes.Structure):
    _fields_ = [("prev", ctypes.c_void_p), ("cur", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("params", Params), ("blob", ctypes.c_void_p), ("blob_cap", ctypes.c_size_t)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("arena", ctypes.c_void_p), ("arena_bytes", ctypes.c_size_t),
                ("slots", ctypes.c_int32), ("max_series", ctypes.c_int32),
                ("dry_run", ctypes.c_int32), ("dry_run_us", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("series", ctypes.c_int32), ("params", Params),
                ("n", ctypes.c_int64), ("host_in", ctypes.c_void_p), ("host_out", ctypes.c_void_p),
                ("host_out_cap", ctypes.c_size_t), ("start", ctypes.c_int64),
                ("count", ctypes.c_int64)]


class Completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("series", ctypes.c_int32), ("reference", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("out_bytes", ctypes.c_uint64), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_end", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("started", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("deferred_memory", ctypes.c_uint64),
                ("arena_bytes", ctypes.c_uint64), ("arena_used", ctypes.c_uint64),
                ("arena_peak", ctypes.c_uint64), ("max_inflight", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("now", ctypes.c_double)]


REQ_COMPRESS = 0
REQ_DECOMPRESS = 1


class BatchDecodeItem(ctypes.Structure):
    _fields_ = [("blob", ctypes.c_void_p), ("prev", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("n", ctypes.c_int64)]


class FusedTuning(ctypes.Structure):
    _fields_ = [("k1_threads", ctypes.c_int32), ("exact_warps", ctypes.c_int32),
                ("decode_seg_log2", ctypes.c_int32), ("groups", ctypes.c_int32),
                ("streams", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def fused_tuning(t=(1024, 8, 0, 1, 1)) -> FusedTuning:
    """(k1_threads, exact_warps, decode_seg_log2[, groups, streams]) as numarck_fused_tuning."""
    t = tuple(int(v) for v in t) + (1, 1)[max(0, len(t) - 3):]
    return FusedTuning(t[0], t[1], t[2], t[3], t[4], 0)


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
        pp = ctypes.POINTER(Params)
        L.numarck_compress_bound.argtypes = [i64, pp]
        L.numarck_compress_bound.restype = sz
        L.numarck_workspace_bytes.argtypes = [i64, pp]
        L.numarck_workspace_bytes.restype = sz
        L.numarck_workspace_init.argtypes = [vp, sz, vp]
        L.numarck_workspace_init.restype = i32
        L.numarck_compress.argtypes = [vp, vp, i64, pp, vp, sz, vp, sz, vp]
        L.numarck_compress.restype = i32
        L.numarck_blob_size.argtypes = [vp, ctypes.POINTER(sz)]
        L.numarck_blob_size.restype = i32
        L.numarck_read_header.argtypes = [vp, vp]
        L.numarck_read_header.restype = i32
        L.numarck_decompress.argtypes = [vp, vp, vp, vp, i64, vp, vp]
        L.numarck_decompress.restype = i32
        L.numarck_decompress_range.argtypes = [vp, vp, vp, i64, i64, vp, vp, vp]
        L.numarck_decompress_range.restype = i32
        L.numarck_decompress_compress.argtypes = [vp, vp, vp, vp, i64, vp, vp, pp, vp, sz, vp, sz,
                                                   vp]
        L.numarck_decompress_compress.restype = i32
        L.numarck_selftest_wait.argtypes = [vp, i64, vp, vp]
        L.numarck_selftest_wait.restype = i32
        L.numarck_status_string.argtypes = [i32]
        L.numarck_status_string.restype = ctypes.c_char_p
        L.numarck_trace_events.argtypes = [ctypes.POINTER(ctypes.c_void_p), i32]
        L.numarck_trace_events.restype = i32
        L.numarck_batch_workspace_bytes.argtypes = [ctypes.POINTER(BatchItem), i32, i32]
        L.numarck_batch_workspace_bytes.restype = sz
        L.numarck_compress_batch.argtypes = [ctypes.POINTER(BatchItem), i32, i32, i32, vp, sz, vp]
        L.numarck_compress_batch.restype = i32
        L.numarck_decompress_batch.argtypes = [ctypes.POINTER(BatchDecodeItem), i32, i32, i32, vp,
                                               vp]
        L.numarck_decompress_batch.restype = i32
        ft = ctypes.POINTER(FusedTuning)
        L.numarck_fused_workspace_bytes.argtypes = [ctypes.POINTER(BatchItem), i32]
        L.numarck_fused_workspace_bytes.restype = sz
        L.numarck_compress_batch_fused.argtypes = [ctypes.POINTER(BatchItem), i32, ft, vp, sz, vp]
        L.numarck_compress_batch_fused.restype = i32
        L.numarck_fused_decode_workspace_bytes.argtypes = [i32]
        L.numarck_fused_decode_workspace_bytes.restype = sz
        L.numarck_decompress_batch_fused.argtypes = [ctypes.POINTER(BatchDecodeItem), i32, ft, vp,
                                                     sz, vp, vp]
        L.numarck_decompress_batch_fused.restype = i32
        L.numarck_compress_noalloc.argtypes = [vp, vp, i64, pp, vp, sz, vp]
        L.numarck_compress_noalloc.restype = i32
        L.numarck_version.argtypes = []
        L.numarck_version.restype = ctypes.c_char_p
        L.numarck_zindex_bound.argtypes = [vp]
        L.numarck_zindex_bound.restype = sz
        L.numarck_zindex_workspace_bytes.argtypes = [vp]
        L.numarck_zindex_workspace_bytes.restype = sz
        L.numarck_deflate_index.argtypes = [vp, vp, vp, sz, vp, sz, vp]
        L.numarck_deflate_index.restype = i32
        L.numarck_inflate_index.argtypes = [vp, sz, vp, vp, i64, i64, vp, vp]
        L.numarck_inflate_index.restype = i32
        L.numarck_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(i32)]
        L.numarck_server_create.restype = vp
        L.numarck_server_submit.argtypes = [vp, ctypes.POINTER(Request),
                                            ctypes.POINTER(ctypes.c_uint64)]
        L.numarck_server_submit.restype = i32
        L.numarck_server_poll.argtypes = [vp, ctypes.POINTER(Completion), i32, ctypes.POINTER(i32),
                                          i32]
        L.numarck_server_poll.restype = i32
        L.numarck_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
        L.numarck_server_get_stats.restype = i32
        L.numarck_server_destroy.argtypes = [vp]
        L.numarck_server_destroy.restype = i32
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().numarck_status_string(int(code)).decode()


def _check(code: int, what: str):
    if code != OK:
        raise NumarckError(code, what)


def make_params(dtype, B: int, E: float, anchor: int = ANCHOR_ZERO, block_bytes: int = 0) -> Params:
    code = {torch.float32: F32, torch.float64: F64}.get(dtype, dtype)
    return Params(int(code), int(B), float(E), int(anchor), 0, int(block_bytes))


def compress_bound(n: int, params: Params) -> int:
    return int(lib().numarck_compress_bound(int(n), ctypes.byref(params)))


def workspace_bytes(n: int, params: Params) -> int:
    return int(lib().numarck_workspace_bytes(int(n), ctypes.byref(params)))


def _stream_ptr(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Workspace:
    """A device workspace, zero-filled once and reused (grows on demand)."""

    def __init__(self, device=None):
        self.device = torch.device(device or "cuda")
        self.buf = None

    def get(self, nbytes: int, stream=None) -> torch.Tensor:
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            _check(lib().numarck_workspace_init(ctypes.c_void_p(self.buf.data_ptr()), nbytes,
                                                ctypes.c_void_p(_stream_ptr(stream))),
                   "numarck_workspace_init")
        return self.buf


_default_ws = {}


def _workspace_for(device) -> Workspace:
    key = torch.device(device).index
    if key not in _default_ws:
        _default_ws[key] = Workspace(device)
    return _default_ws[key]


def compress(prev: torch.Tensor, cur: torch.Tensor, E: float, B: int, anchor: int = ANCHOR_ZERO,
             block_bytes: int = 0, blob: torch.Tensor | None = None,
             workspace: Workspace | None = None, stream=None) -> torch.Tensor:
    """Queues compression of `cur` against `prev` (1-D CUDA tensors of equal dtype/length).

    Returns the blob buffer (uint8, compress_bound bytes); its header says how many bytes are
    used (see header()/blob_size())."""
    if prev.dtype != cur.dtype or prev.shape != cur.shape or prev.dim() != 1:
        raise ValueError("prev and cur must be 1-D tensors of the same dtype and length")
    if not (prev.is_cuda and cur.is_cuda):
        raise ValueError("prev and cur must be CUDA tensors")
    prev = prev.contiguous()
    cur = cur.contiguous()
    params = make_params(prev.dtype, B, E, anchor, block_bytes)
    n = prev.numel()
    bound = compress_bound(n, params)
    if bound == 0:
        raise NumarckError(ERR_INVALID_ARG, "numarck_compress_bound")
    if blob is None:
        blob = torch.empty(bound, dtype=torch.uint8, device=prev.device)
    ws = (workspace or _workspace_for(prev.device)).get(workspace_bytes(n, params), stream)
    _check(lib().numarck_compress(ctypes.c_void_p(prev.data_ptr()), ctypes.c_void_p(cur.data_ptr()),
                                  n, ctypes.byref(params), ctypes.c_void_p(blob.data_ptr()),
                                  blob.numel(), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                  ctypes.c_void_p(_stream_ptr(stream))), "numarck_compress")
    return blob


def header_bytes(blob: torch.Tensor) -> bytes:
    """Host copy of the blob header (synchronises with the current stream)."""
    return bytes(blob[:HEADER_BYTES].cpu().numpy().tobytes())


def parse_header(hb: bytes) -> dict:
    size = struct.calcsize(_HEADER_FMT)
    return dict(zip(HEADER_FIELDS, struct.unpack(_HEADER_FMT, hb[:size])))


def blob_size(hb: bytes) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().numarck_blob_size(ctypes.c_char_p(hb), ctypes.byref(out)), "numarck_blob_size")
    return int(out.value)


def decompress(blob: torch.Tensor, prev: torch.Tensor, header: bytes | None = None,
               out: torch.Tensor | None = None, status: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
    prev = prev.contiguous()
    if out is None:
        out = torch.empty_like(prev)
    hp = ctypes.c_char_p(header) if header is not None else None
    sp = ctypes.c_void_p(status.data_ptr()) if status is not None else None
    _check(lib().numarck_decompress(ctypes.c_void_p(blob.data_ptr()), hp,
                                    ctypes.c_void_p(prev.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                    prev.numel(), sp, ctypes.c_void_p(_stream_ptr(stream))),
           "numarck_decompress")
    return out


def decompress_range(blob: torch.Tensor, prev_seg: torch.Tensor, start: int, count: int,
                     header: bytes | None = None, out: torch.Tensor | None = None,
                     status: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    prev_seg = prev_seg.contiguous()
    if out is None:
        out = torch.empty_like(prev_seg)
    hp = ctypes.c_char_p(header) if header is not None else None
    sp = ctypes.c_void_p(status.data_ptr()) if status is not None else None
    _check(lib().numarck_decompress_range(ctypes.c_void_p(blob.data_ptr()), hp,
                                          ctypes.c_void_p(prev_seg.data_ptr()), int(start),
                                          int(count), ctypes.c_void_p(out.data_ptr()), sp,
                                          ctypes.c_void_p(_stream_ptr(stream))),
           "numarck_decompress_range")
    return out


def decompress_compress(blob: torch.Tensor, prev: torch.Tensor, next_cur: torch.Tensor, E: float,
                        B: int, anchor: int = ANCHOR_ZERO, block_bytes: int = 0,
                        out: torch.Tensor | None = None, next_blob: torch.Tensor | None = None,
                        workspace: Workspace | None = None, status: torch.Tensor | None = None,
                        header: bytes | None = None, stream=None):
    """One step of a chain of timesteps: decompresses `blob` (compressed against `prev`) into
    `out` and queues the compression of `next_cur` against `out` into `next_blob`
    (numarck_decompress_compress). Returns (out, next_blob)."""
    if prev.dtype != next_cur.dtype or prev.shape != next_cur.shape or prev.dim() != 1:
        raise ValueError("prev and next_cur must be 1-D tensors of the same dtype and length")
    if not (prev.is_cuda and next_cur.is_cuda and blob.is_cuda):
        raise ValueError("blob, prev and next_cur must be CUDA tensors")
    prev = prev.contiguous()
    next_cur = next_cur.contiguous()
    params = make_params(prev.dtype, B, E, anchor, block_bytes)
    n = prev.numel()
    bound = compress_bound(n, params)
    if bound == 0:
        raise NumarckError(ERR_INVALID_ARG, "numarck_compress_bound")
    if out is None:
        out = torch.empty_like(prev)
    if next_blob is None:
        next_blob = torch.empty(bound, dtype=torch.uint8, device=prev.device)
    ws = (workspace or _workspace_for(prev.device)).get(workspace_bytes(n, params), stream)
    hp = ctypes.c_char_p(header) if header is not None else None
    sp = ctypes.c_void_p(status.data_ptr()) if status is not None else None
    _check(lib().numarck_decompress_compress(
        ctypes.c_void_p(blob.data_ptr()), hp, ctypes.c_void_p(prev.data_ptr()),
        ctypes.c_void_p(out.data_ptr()), n, sp, ctypes.c_void_p(next_cur.data_ptr()),
        ctypes.byref(params), ctypes.c_void_p(next_blob.data_ptr()), next_blob.numel(),
        ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.c_void_p(_stream_ptr(stream))),
        "numarck_decompress_compress")
    return out, next_blob


class Chain:
    """A chain of timesteps of one variable compressed as the paper's in-situ use does (Eq. 4:
    each timestep against the reconstruction of the previous one), through the chained step.

    push(x) takes the next timestep (a 1-D CUDA tensor of the chain's dtype and length). The
    first push only keeps x as the reference. Every later push returns the blob of x (a view of
    an internal buffer, valid until the push after next); from the third push on, the
    reconstruction of the previous timestep is made by the same call that compresses x
    (numarck_decompress_compress). reconstruction() returns the reconstruction of the latest
    timestep (decompressing the latest blob if the next push has not made it yet)."""

    def __init__(self, n: int, dtype, E: float, B: int, anchor: int = ANCHOR_ZERO,
                 block_bytes: int = 0, device="cuda", stream=None):
        self.n, self.dtype, self.E, self.B = int(n), dtype, float(E), int(B)
        self.anchor, self.block_bytes, self.stream = anchor, block_bytes, stream
        params = make_params(dtype, B, E, anchor, block_bytes)
        bound = compress_bound(self.n, params)
        if bound == 0:
            raise NumarckError(ERR_INVALID_ARG, "numarck_compress_bound")
        dev = torch.device(device)
        self.blobs = [torch.empty(bound, dtype=torch.uint8, device=dev) for _ in range(2)]
        self.recs = [torch.empty(self.n, dtype=dtype, device=dev) for _ in range(2)]
        self.ws = Workspace(dev)
        self.ws.get(workspace_bytes(self.n, params), stream)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.ref = None          # the first timestep (the prev of the first blob)
        self.base = None         # the prev the latest blob was compressed against
        self.latest = -1         # index of the blob buffer holding the latest blob
        self.recon = None        # reconstruction of the latest timestep, once made
        self.t = 0               # timesteps pushed

    def push(self, x: torch.Tensor):
        if x.dtype != self.dtype or x.numel() != self.n or x.dim() != 1 or not x.is_cuda:
            raise ValueError("a timestep must be a 1-D CUDA tensor of the chain's dtype and length")
        kw = dict(anchor=self.anchor, block_bytes=self.block_bytes, workspace=self.ws,
                  stream=self.stream)
        self.t += 1
        if self.t == 1:
            self.ref = x.clone()
            self.recon = self.ref
            return None
        nxt = 0 if self.latest != 0 else 1
        if self.t == 2:
            compress(self.ref, x, self.E, self.B, blob=self.blobs[nxt], **kw)
            self.base = self.ref
        else:
            # the reconstruction of the previous timestep, made while compressing x against it
            out = self._free_rec()
            decompress_compress(self.blobs[self.latest], self.base, x, self.E, self.B, out=out,
                                next_blob=self.blobs[nxt], status=self.status, **kw)
            self.base = out
        self.latest = nxt
        self.recon = None
        return self.blobs[nxt]

    def _free_rec(self) -> torch.Tensor:
        # the reconstruction buffer that is not the base of the latest blob
        return self.recs[1] if self.base is self.recs[0] else self.recs[0]

    def reconstruction(self) -> torch.Tensor:
        if self.recon is None:
            self.recon = decompress(self.blobs[self.latest], self.base, out=self._free_rec(),
                                    status=self.status, stream=self.stream)
        return self.recon

    def check(self) -> int:
        """The device status word of the chain's decompressions (synchronises)."""
        return int(self.status.item())


def selftest_wait(flag: torch.Tensor, limit_ns: int, status: torch.Tensor, stream=None) -> None:
    """Queues the library's bounded device wait on `flag` (an int64 CUDA tensor): `status`
    (int32 CUDA tensor) receives OK if the flag is non-zero within limit_ns, else ERR_TIMEOUT
    (numarck_selftest_wait)."""
    _check(lib().numarck_selftest_wait(ctypes.c_void_p(flag.data_ptr()), int(limit_ns),
                                       ctypes.c_void_p(status.data_ptr()),
                                       ctypes.c_void_p(_stream_ptr(stream))),
           "numarck_selftest_wait")


class Batch:
    """A fixed list of variables to compress together.

    pairs: list of (prev, cur) 1-D CUDA tensors; specs: list of (E, B) or (E, B, anchor,
    block_bytes) per variable. Blob buffers are allocated once (compress_bound bytes each) and
    reused by every run, so a run can be captured into a CUDA graph.

    Two ways to run it, with the same results: "lanes" (numarck_compress_batch: each variable's
    kernels, `lanes` variables in flight, grids sized for 1/grid_share of the GPU) and "fused"
    (numarck_compress_batch_fused: one launch per phase over all variables; `tuning` is
    (k1_threads, exact_warps, decode_seg_log2, groups, streams)). Each way keeps its own
    workspace, zero-filled again whenever its layout (the lane count) changes."""

    def __init__(self, pairs, specs, lanes=8, grid_share=4, workspace=None, mode="lanes",
                 tuning=(1024, 8, 0, 1, 1)):
        self.pairs = [(p.contiguous(), x.contiguous()) for p, x in pairs]
        self.lanes, self.grid_share = int(lanes), int(grid_share)
        self.mode = mode
        self.tuning = tuple(tuning)
        arr = (BatchItem * len(pairs))()
        self.blobs = []
        for i, ((p, x), spec) in enumerate(zip(self.pairs, specs)):
            E, B = spec[0], spec[1]
            anchor = spec[2] if len(spec) > 2 else ANCHOR_ZERO
            bb = spec[3] if len(spec) > 3 else 0
            prm = make_params(p.dtype, B, E, anchor, bb)
            bound = compress_bound(p.numel(), prm)
            if bound == 0:
                raise NumarckError(ERR_INVALID_ARG, f"batch item {i}")
            blob = torch.empty(bound, dtype=torch.uint8, device=p.device)
            self.blobs.append(blob)
            arr[i] = BatchItem(p.data_ptr(), x.data_ptr(), p.numel(), prm, blob.data_ptr(), bound)
        self.items = arr
        self.count = len(pairs)
        dev = self.pairs[0][0].device if self.pairs else "cuda"
        self.ws = workspace or Workspace(dev)
        self.fws = Workspace(dev)
        self.dws = None
        self._lane_layout = None

    def set_lanes(self, lanes, grid_share):
        self.mode = "lanes"
        self.lanes, self.grid_share = int(lanes), int(grid_share)

    def set_fused(self, tuning=(1024, 8, 0, 1, 1)):
        self.mode = "fused"
        self.tuning = tuple(tuning)

    def _tuning(self):
        return fused_tuning(self.tuning)

    def run(self, stream=None):
        """Queues the compression of every variable; returns the list of blob buffers."""
        if self.mode == "fused":
            need = int(lib().numarck_fused_workspace_bytes(self.items, self.count))
            if need == 0 and self.count:
                raise NumarckError(ERR_INVALID_ARG, "numarck_fused_workspace_bytes")
            ws = self.fws.get(need, stream)
            t = self._tuning()
            _check(lib().numarck_compress_batch_fused(self.items, self.count, ctypes.byref(t),
                                                      ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                                      ctypes.c_void_p(_stream_ptr(stream))),
                   "numarck_compress_batch_fused")
            return self.blobs
        need = int(lib().numarck_batch_workspace_bytes(self.items, self.count, self.lanes))
        if need == 0 and self.count:
            raise NumarckError(ERR_INVALID_ARG, "numarck_batch_workspace_bytes")
        fresh = self.ws.buf is None or self.ws.buf.numel() < need
        ws = self.ws.get(need, stream)
        if not fresh and self._lane_layout not in (None, self.lanes):
            # another lane count placed the lanes' slices elsewhere: start from zero again
            _check(lib().numarck_workspace_init(ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                                ctypes.c_void_p(_stream_ptr(stream))),
                   "numarck_workspace_init")
        self._lane_layout = self.lanes
        _check(lib().numarck_compress_batch(self.items, self.count, self.lanes, self.grid_share,
                                            ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                            ctypes.c_void_p(_stream_ptr(stream))),
               "numarck_compress_batch")
        return self.blobs

    def decompress(self, prevs, outs=None, status=None, stream=None):
        """Reconstructs every variable from this batch's blobs, the same way the batch runs."""
        if self.mode != "fused":
            return decompress_batch(self.blobs, prevs, outs=outs, lanes=self.lanes,
                                    grid_share=self.grid_share, status=status, stream=stream)
        if self.dws is None:
            nbytes = int(lib().numarck_fused_decode_workspace_bytes(self.count))
            self.dws = torch.empty(max(nbytes, 256), dtype=torch.uint8,
                                   device=self.blobs[0].device)
        return decompress_batch_fused(self.blobs, prevs, outs=outs, tuning=self.tuning,
                                      workspace=self.dws, status=status, stream=stream)


def decompress_batch_fused(blobs, prevs, outs=None, tuning=(1024, 8, 0, 1, 1), workspace=None,
                           status=None, stream=None):
    """numarck_decompress_batch_fused: every blob of a batch in one prep and one decode launch."""
    outs = outs or [torch.empty_like(p) for p in prevs]
    arr = (BatchDecodeItem * len(blobs))()
    for i, (b, p, o) in enumerate(zip(blobs, prevs, outs)):
        arr[i] = BatchDecodeItem(b.data_ptr(), p.data_ptr(), o.data_ptr(), p.numel())
    if workspace is None:
        nbytes = int(lib().numarck_fused_decode_workspace_bytes(len(blobs)))
        workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=blobs[0].device)
    t = fused_tuning(tuning)
    sp = ctypes.c_void_p(status.data_ptr()) if status is not None else None
    _check(lib().numarck_decompress_batch_fused(arr, len(blobs), ctypes.byref(t),
                                                ctypes.c_void_p(workspace.data_ptr()),
                                                workspace.numel(), sp,
                                                ctypes.c_void_p(_stream_ptr(stream))),
           "numarck_decompress_batch_fused")
    return outs


def decompress_batch(blobs, prevs, outs=None, lanes=8, grid_share=4, status=None, stream=None):
    """Reconstructs every variable of a batch (one blob and one prev per variable)."""
    outs = outs or [torch.empty_like(p) for p in prevs]
    arr = (BatchDecodeItem * len(blobs))()
    for i, (b, p, o) in enumerate(zip(blobs, prevs, outs)):
        arr[i] = BatchDecodeItem(b.data_ptr(), p.data_ptr(), o.data_ptr(), p.numel())
    sp = ctypes.c_void_p(status.data_ptr()) if status is not None else None
    _check(lib().numarck_decompress_batch(arr, len(blobs), int(lanes), int(grid_share), sp,
                                          ctypes.c_void_p(_stream_ptr(stream))),
           "numarck_decompress_batch")
    return outs


def compress_noalloc(prev, cur, E, B, anchor=ANCHOR_ZERO, block_bytes=0, blob=None, stream=None):
    """numarck_compress_noalloc: compression without a caller workspace (static scratch)."""
    params = make_params(prev.dtype, B, E, anchor, block_bytes)
    if blob is None:
        blob = torch.empty(compress_bound(prev.numel(), params), dtype=torch.uint8,
                           device=prev.device)
    _check(lib().numarck_compress_noalloc(ctypes.c_void_p(prev.data_ptr()),
                                          ctypes.c_void_p(cur.data_ptr()), prev.numel(),
                                          ctypes.byref(params), ctypes.c_void_p(blob.data_ptr()),
                                          blob.numel(), ctypes.c_void_p(_stream_ptr(stream))),
           "numarck_compress_noalloc")
    return blob


_trace_keep = None


def trace_events(events) -> None:
    """Record these torch.cuda.Event objects at the kernel boundaries of the following calls on
    this thread (see numarck_trace_events); None stops recording."""
    global _trace_keep
    if events is None:
        _trace_keep = None
        _check(lib().numarck_trace_events(None, 0), "numarck_trace_events")
        return
    arr = (ctypes.c_void_p * len(events))(*[ctypes.c_void_p(e.cuda_event) for e in events])
    _trace_keep = arr
    _check(lib().numarck_trace_events(arr, len(events)), "numarck_trace_events")


def version() -> str:
    return lib().numarck_version().decode()


ZINDEX_HEADER_BYTES = 64
_ZINDEX_FMT = "<Iiiiqqqqqq"
ZINDEX_FIELDS = ("magic", "version", "B", "pad", "n", "nblocks", "nsub", "off_zoff", "off_sub_zoff",
                 "off_data")


def deflate_index(blob: torch.Tensor, header: bytes, zindex: torch.Tensor | None = None,
                  workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Lossless compression of the blob's index blocks into a container of zlib streams
    (numarck_deflate_index); returns the container buffer (its size: zindex_size)."""
    hp = ctypes.c_char_p(header)
    if zindex is None:
        zindex = torch.empty(lib().numarck_zindex_bound(hp), dtype=torch.uint8, device=blob.device)
    if workspace is None:
        workspace = torch.empty(lib().numarck_zindex_workspace_bytes(hp), dtype=torch.uint8,
                                device=blob.device)
    _check(lib().numarck_deflate_index(ctypes.c_void_p(blob.data_ptr()), hp,
                                       ctypes.c_void_p(zindex.data_ptr()), zindex.numel(),
                                       ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                       ctypes.c_void_p(_stream_ptr(stream))), "numarck_deflate_index")
    return zindex


def zindex_header(zindex: torch.Tensor) -> dict:
    """The container header, with the container's size (zoff[nblocks]) as 'total_bytes'
    (synchronises with the current stream)."""
    raw = bytes(zindex[:ZINDEX_HEADER_BYTES].cpu().numpy().tobytes())
    h = dict(zip(ZINDEX_FIELDS, struct.unpack(_ZINDEX_FMT, raw)))
    at = h["off_zoff"] + 8 * h["nblocks"]
    h["total_bytes"] = int(zindex[at:at + 8].cpu().view(torch.int64).item())
    return h


def zindex_offsets(zindex: torch.Tensor, h: dict):
    """(zoff[nblocks + 1], sub_zoff[nsub]) as numpy arrays (host copies)."""
    zo = zindex[h["off_zoff"]:h["off_zoff"] + 8 * (h["nblocks"] + 1)].cpu().view(torch.int64)
    so = zindex[h["off_sub_zoff"]:h["off_sub_zoff"] + 8 * h["nsub"]].cpu().view(torch.int64)
    return zo.numpy(), so.numpy()


def inflate_index(zindex: torch.Tensor, zbytes: int, header: bytes, blob: torch.Tensor,
                  start: int = 0, count: int | None = None, status: torch.Tensor | None = None,
                  stream=None) -> None:
    """Restores the index sub-blocks covering [start, start + count) into `blob`."""
    n = parse_header(header)["n"]
    cnt = n - start if count is None else count
    sp = ctypes.c_void_p(status.data_ptr()) if status is not None else None
    _check(lib().numarck_inflate_index(ctypes.c_void_p(zindex.data_ptr()), int(zbytes),
                                       ctypes.c_char_p(header), ctypes.c_void_p(blob.data_ptr()),
                                       int(start), int(cnt), sp,
                                       ctypes.c_void_p(_stream_ptr(stream))), "numarck_inflate_index")


class Server:
    """The served form (numarck_server_*): a request loop over resident time series in one
    device arena. Host buffers passed to submit() must be pinned and stay alive until their
    completion is polled (this object keeps a reference until then)."""

    def __init__(self, arena: torch.Tensor | None, slots: int = 8, max_series: int = 64,
                 dry_run_us: int | None = None, arena_bytes: int | None = None):
        size = arena.numel() if arena is not None else (arena_bytes or (1 << 40))
        cfg = ServerConfig(ctypes.c_void_p(arena.data_ptr() if arena is not None else 0), size,
                           int(slots),
                           int(max_series), 1 if dry_run_us is not None else 0,
                           int(dry_run_us or 0))
        st = ctypes.c_int32(0)
        self._arena = arena
        self._h = lib().numarck_server_create(ctypes.byref(cfg), ctypes.byref(st))
        if not self._h:
            raise NumarckError(st.value, "numarck_server_create")
        self._keep = {}

    def submit(self, kind: int, series: int, n: int, params: Params | None = None,
               host_in: torch.Tensor | None = None, host_out: torch.Tensor | None = None,
               start: int = 0, count: int | None = None) -> int:
        r = Request(int(kind), int(series), params or Params(), int(n),
                    ctypes.c_void_p(host_in.data_ptr() if host_in is not None else 0),
                    ctypes.c_void_p(host_out.data_ptr() if host_out is not None else 0),
                    host_out.numel() * host_out.element_size() if host_out is not None else 0,
                    int(start), int(n - start if count is None else count))
        rid = ctypes.c_uint64(0)
        _check(lib().numarck_server_submit(self._h, ctypes.byref(r), ctypes.byref(rid)),
               "numarck_server_submit")
        self._keep[rid.value] = (host_in, host_out)
        return rid.value

    def poll(self, max_items: int = 256, wait_ms: int = 0) -> list:
        arr = (Completion * max_items)()
        got = ctypes.c_int32(0)
        _check(lib().numarck_server_poll(self._h, arr, max_items, ctypes.byref(got), int(wait_ms)),
               "numarck_server_poll")
        out = []
        for i in range(got.value):
            c = arr[i]
            self._keep.pop(c.id, None)
            out.append({f: getattr(c, f) for f, _ in Completion._fields_ if f != "pad"})
        return out

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().numarck_server_get_stats(self._h, ctypes.byref(st)), "numarck_server_get_stats")
        return {f: getattr(st, f) for f, _ in ServerStats._fields_ if f != "pad"}

    def close(self) -> None:
        if self._h:
            h, self._h = self._h, None
            _check(lib().numarck_server_destroy(h), "numarck_server_destroy")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
