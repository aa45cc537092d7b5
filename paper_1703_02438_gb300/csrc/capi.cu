// capi.cu — the extern "C" boundary of the NUMARCK library (declared in include/numarck.h).
//
// Host side only: argument validation, blob geometry (§IV.C block layout, §IV.D arrays),
// workspace layout, and the launch sequence K0 (ANCHOR_MIN) -> K1 -> K2 -> K3a -> K3b -> K3c for
// compression and K4 for (partial) decompression. Nothing here allocates device memory.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>

#include "launch.h"

using namespace nmk;

namespace {

int64_t round_up(int64_t x, int64_t m) { return round_up_i64(x, m); }

// float nearest to v rounded toward -inf / +inf
float f_down(double v) {
  float f = (float)v;
  if ((double)f > v) f = std::nextafter(f, -INFINITY);
  return f;
}
float f_up(double v) {
  float f = (float)v;
  if ((double)f < v) f = std::nextafter(f, INFINITY);
  return f;
}

int check_params(const numarck_params* p) {
  if (!p) return NUMARCK_ERR_INVALID_ARG;
  if (p->dtype != NUMARCK_F32 && p->dtype != NUMARCK_F64) return NUMARCK_ERR_INVALID_ARG;
  if (p->B < 0 || p->B > NUMARCK_MAX_B) return NUMARCK_ERR_INVALID_ARG;   // 0: automatic
  if (!std::isfinite(p->E) || !(p->E >= 0x1p-60) || !(p->E < 1.0)) return NUMARCK_ERR_INVALID_ARG;
  if (p->anchor != NUMARCK_ANCHOR_ZERO && p->anchor != NUMARCK_ANCHOR_MIN)
    return NUMARCK_ERR_INVALID_ARG;
  if (p->reserved != 0) return NUMARCK_ERR_INVALID_ARG;
  if (p->block_bytes != 0 && (p->block_bytes < 2 || p->block_bytes > ((int64_t)1 << 30)))
    return NUMARCK_ERR_INVALID_ARG;
  return NUMARCK_OK;
}

// Geometry a call needs room for. For B = 0 (chosen after the histogram) it must cover every
// B = 1..16: off_exact is the largest over B (so the blob bound and K1's code area fit any
// layout) and nsub the largest over B (index blocks of any B end in a partial tile, so a
// smaller B can have more sub-blocks); the other fields are those of B = 16.
Geometry room_geometry(int64_t n, const numarck_params* p, int64_t bb) {
  if (p->B) return make_geometry(n, p->dtype, p->B, bb, p->anchor);
  Geometry g = make_geometry(n, p->dtype, NUMARCK_MAX_B, bb, p->anchor);
  for (int B = 1; B < NUMARCK_MAX_B; ++B) {
    const Geometry h = make_geometry(n, p->dtype, B, bb, p->anchor);
    g.off_exact = std::max(g.off_exact, h.off_exact);
    g.nsub = std::max(g.nsub, h.nsub);
  }
  return g;
}

int64_t effective_block_bytes(const numarck_params* p) {
  return p->block_bytes ? p->block_bytes : (int64_t)NUMARCK_DEFAULT_BLOCK_BYTES;
}

WsLayout make_ws(const Geometry& g) {
  WsLayout w{};
  size_t o = 0;
  w.ctrl = o;
  o += sizeof(Ctrl);
  w.hist = o;
  o = (size_t)round_up((int64_t)(o + (size_t)HWIN * 8), 256);
  w.rank = o;
  o = (size_t)round_up((int64_t)(o + (size_t)HWIN * 2), 256);
  w.mtab = o;
  o += (size_t)65536 * 8;
  w.cftab = o;
  o += (size_t)65536 * 4;
  w.selb = o;
  o += (size_t)65536 * 4;
  w.status = o;   // per-tile incompressible counts, then the offset scan's look-back flags
  o = (size_t)round_up((int64_t)(o + (size_t)(g.nsub + g.nsub / 4096 + 2) * 8), 256);
  w.total = o;
  return w;
}

template <typename T>
Consts<T> make_consts(double E, int anchor) {
  Consts<T> c{};
  c.E_T = (T)E;
  c.w = c.E_T + c.E_T;
  c.inv_w = (T)1 / c.w;
  c.cap = c.w * (T)(1 << WIN_LOG2);
  c.a = anchor == NUMARCK_ANCHOR_ZERO ? -c.E_T : (T)0;
  c.hbase = anchor == NUMARCK_ANCHOR_ZERO ? -((1 << WIN_LOG2) + HMARGIN) : -HMARGIN;
  c.af = (float)c.a;
  c.inv_wf = (float)c.inv_w;
  c.Ef = (float)c.E_T;
  c.wf = (float)c.w;
  c.cap_lo = f_down(std::fmin((double)c.cap * (1.0 - 0x1p-19), 0x1p100));
  c.cap_hi = f_up((double)c.cap * (1.0 + 0x1p-19));
  c.K0 = f_up(0x1p-19 * (double)c.inv_w * std::fabs((double)c.a) + 0x1p-60);
  c.kA = f_up((0x1p-22 + 0x1p-23 + 0x1p-50) * (1.0 + 0x1p-40));
  c.k1 = f_up(0x1p-20 * (1.0 + (double)c.Ef) * (1.0 + 0x1p-40));
  c.C0 = f_up((0x1p-22 * std::fabs((double)c.af) + 0x1p-49 + 0x1p-50 + 0x1p-100) * (1.0 + 0x1p-40));
  return c;
}

int device_sms() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (dev < 64 && cache[dev]) return cache[dev];
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (dev < 64) cache[dev] = sms;
  return sms;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

thread_local void* const* g_trace = nullptr;
thread_local int g_trace_count = 0;

void trace(int i, int need, cudaStream_t s) { trace_event(i, need, s); }

int decode(const void* blob, const void* header_host, const void* prev_seg, int64_t start,
           int64_t count, void* out_seg, int64_t n_expected, int32_t* status_dev,
           numarck_stream_t stream) {
  if (!blob || !aligned(blob, 256)) return NUMARCK_ERR_INVALID_ARG;
  if (count < 0 || start < 0) return NUMARCK_ERR_RANGE;
  int64_t ntiles = 0;
  if (header_host) {
    numarck_header h;
    std::memcpy(&h, header_host, sizeof(h));
    Geometry g;
    const int rc = check_header(h, &g);
    if (rc) return rc;
    if (n_expected >= 0 && n_expected != h.n) return NUMARCK_ERR_INVALID_ARG;
    if (start > h.n || count > h.n - start) return NUMARCK_ERR_RANGE;
    if (count == 0) return NUMARCK_OK;
    const size_t L = h.dtype == NUMARCK_F64 ? 8 : 4;
    if (!prev_seg || !out_seg || !aligned(prev_seg, L) || !aligned(out_seg, L))
      return NUMARCK_ERR_INVALID_ARG;
    const int64_t first = start, last = start + count - 1;
    const int64_t q0 = first / g.epb, q1 = last / g.epb;
    ntiles = (q1 * g.spb + (last - q1 * g.epb) / SUB) - (q0 * g.spb + (first - q0 * g.epb) / SUB) + 1;
  } else {
    if (count == 0) return NUMARCK_OK;
    if (!prev_seg || !out_seg || !aligned(prev_seg, 4) || !aligned(out_seg, 4))
      return NUMARCK_ERR_INVALID_ARG;
  }
  DecodePlan P{};
  P.blob = static_cast<const unsigned char*>(blob);
  P.prev_seg = prev_seg;
  P.out_seg = out_seg;
  P.status = status_dev;
  P.start = start;
  P.count = count;
  P.n_expected = n_expected;
  P.ntiles_hint = ntiles;
  P.sms = device_sms();
  if (P.sms <= 0) return NUMARCK_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  trace(0, 2, s);
  if (launch_decode(P, s) != cudaSuccess) return NUMARCK_ERR_CUDA;
  trace(1, 2, s);
  return NUMARCK_OK;
}

}  // namespace

extern "C" {

size_t numarck_compress_bound(int64_t n, const numarck_params* p) {
  if (check_params(p) || n < 0 || n > MAX_N) return 0;
  const Geometry g = room_geometry(n, p, effective_block_bytes(p));
  return (size_t)(g.off_exact + n * (p->dtype == NUMARCK_F64 ? 8 : 4));
}

size_t numarck_workspace_bytes(int64_t n, const numarck_params* p) {
  if (check_params(p) || n < 0 || n > MAX_N) return 0;
  return make_ws(room_geometry(n, p, effective_block_bytes(p))).total;
}

int numarck_workspace_init(void* ws, size_t ws_bytes, numarck_stream_t stream) {
  if (!ws) return NUMARCK_ERR_INVALID_ARG;
  if (cudaMemsetAsync(ws, 0, ws_bytes, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
    return NUMARCK_ERR_CUDA;
  return NUMARCK_OK;
}

}  // extern "C"

namespace nmk {

void trace_event(int i, int need, cudaStream_t s) {
  if (g_trace && g_trace_count >= need && g_trace[i])
    cudaEventRecord(static_cast<cudaEvent_t>(g_trace[i]), s);
}

// Validates the arguments of one compression and fills its launch plan (no device access).
int plan_compress(const void* prev, const void* cur, int64_t n, const numarck_params* p,
                  void* blob, size_t blob_cap, void* ws, size_t ws_bytes, CompressPlan* out) {
  int rc = check_params(p);
  if (rc) return rc;
  if (n < 0 || n > MAX_N) return NUMARCK_ERR_INVALID_ARG;
  if (!blob || !ws || !aligned(blob, 256) || !aligned(ws, 256)) return NUMARCK_ERR_INVALID_ARG;
  const size_t L = p->dtype == NUMARCK_F64 ? 8 : 4;
  if (n > 0 && (!prev || !cur || !aligned(prev, L) || !aligned(cur, L)))
    return NUMARCK_ERR_INVALID_ARG;
  const int64_t bb = effective_block_bytes(p);
  // for B = 0 only K0, K1 and the choice of B run on this geometry (K1 uses n, nsub and the
  // code offset); the rest is planned again with the chosen B
  const Geometry g = room_geometry(n, p, bb);
  const WsLayout wl = make_ws(g);
  if (blob_cap < (size_t)(g.off_exact + n * (int64_t)L)) return NUMARCK_ERR_CAPACITY;
  if (ws_bytes < wl.total) return NUMARCK_ERR_CAPACITY;

  CompressPlan& P = *out;
  P = CompressPlan{};
  P.prev = prev;
  P.cur = cur;
  P.blob = static_cast<unsigned char*>(blob);
  P.ws = static_cast<unsigned char*>(ws);
  P.wl = wl;
  P.g = g;
  P.aligned16 = aligned(prev, 16) && aligned(cur, 16);
  P.code_off = code_offset(g);
  P.auto_b = p->B == 0;
  if (p->dtype == NUMARCK_F64)
    P.cd = make_consts<double>(p->E, p->anchor);
  else
    P.cf = make_consts<float>(p->E, p->anchor);

  P.hdr = make_header(g, p->E, bb);
  return NUMARCK_OK;
}

// Queues the kernels of a planned compression that follow K1 (its histogram, codes and bin
// range are complete on stream s).
int launch_compress_tail(const CompressPlan& P0, cudaStream_t s) {
  trace(1, 6, s);
  CompressPlan P = P0;
  if (P0.auto_b) {
    // B from the histogram (§IV.B.2): the geometry of everything after K1 depends on it, so
    // the host reads it back (one synchronisation) and plans the rest with it; K1's codes stay
    // where the B = 16 layout put them (inside every layout's incompressible capacity)
    if (launch_auto_b(P0, s) != cudaSuccess) return NUMARCK_ERR_CUDA;
    int B = 0;
    const Ctrl* ctrl = reinterpret_cast<const Ctrl*>(P0.ws + P0.wl.ctrl);
    if (cudaMemcpyAsync(&B, &ctrl->auto_B, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return NUMARCK_ERR_CUDA;
    if (B < 1 || B > NUMARCK_MAX_B) return NUMARCK_ERR_CUDA;
    numarck_params q{};
    q.dtype = P0.g.dtype;
    q.B = B;
    q.E = P0.hdr.E;
    q.anchor = P0.g.anchor;
    q.block_bytes = P0.hdr.block_bytes;
    size_t cap = (size_t)(P0.g.off_exact + P0.g.n * (P0.g.dtype == NUMARCK_F64 ? 8 : 4));
    const int rc = plan_compress(P0.prev, P0.cur, P0.g.n, &q, P0.blob, cap, P0.ws, P0.wl.total, &P);
    if (rc) return rc;
    P.sms = P0.sms;
    P.code_off = P0.code_off;
  }
  if (launch_topk(P, s) != cudaSuccess) return NUMARCK_ERR_CUDA;
  trace(2, 6, s);
  if (launch_assign(P, s) != cudaSuccess) return NUMARCK_ERR_CUDA;
  trace(3, 6, s);
  if (launch_offsets(P, s) != cudaSuccess) return NUMARCK_ERR_CUDA;
  trace(4, 6, s);
  if (launch_exact(P, s) != cudaSuccess) return NUMARCK_ERR_CUDA;
  trace(5, 6, s);
  return NUMARCK_OK;
}

// Queues the kernels of a planned compression on stream s (P.sms must be set).
int launch_compress(const CompressPlan& P0, cudaStream_t s) {
  trace(0, 6, s);
  if (P0.g.anchor == NUMARCK_ANCHOR_MIN && launch_anchor_min(P0, s) != cudaSuccess)
    return NUMARCK_ERR_CUDA;
  if (launch_hist(P0, s) != cudaSuccess) return NUMARCK_ERR_CUDA;
  return launch_compress_tail(P0, s);
}

int current_device_sms() { return device_sms(); }

int plan_decompress_check(const void* blob, const void* prev, void* out, int64_t n) {
  if (!blob || !aligned(blob, 256) || n < 0) return NUMARCK_ERR_INVALID_ARG;
  if (n > 0 && (!prev || !out || !aligned(prev, 4) || !aligned(out, 4))) return NUMARCK_ERR_INVALID_ARG;
  return NUMARCK_OK;
}

int launch_decompress(const void* blob, const void* prev, void* out, int64_t n, int32_t* status,
                      int sms, cudaStream_t s, int concurrency) {
  if (n == 0) return NUMARCK_OK;
  DecodePlan P{};
  P.blob = static_cast<const unsigned char*>(blob);
  P.prev_seg = prev;
  P.out_seg = out;
  P.status = status;
  P.start = 0;
  P.count = n;
  P.n_expected = n;
  P.ntiles_hint = 0;
  P.sms = sms;
  P.concurrency = concurrency;
  trace(0, 2, s);
  if (launch_decode(P, s) != cudaSuccess) return NUMARCK_ERR_CUDA;
  trace(1, 2, s);
  return NUMARCK_OK;
}

}  // namespace nmk

extern "C" {

int numarck_compress(const void* prev, const void* cur, int64_t n, const numarck_params* p,
                     void* blob, size_t blob_cap, void* ws, size_t ws_bytes,
                     numarck_stream_t stream) {
  nmk::NvtxRange nvtx_("numarck_compress");
  CompressPlan P;
  const int rc = plan_compress(prev, cur, n, p, blob, blob_cap, ws, ws_bytes, &P);
  if (rc) return rc;
  if (P.auto_b) {   // choosing B synchronises the stream once: not allowed while capturing
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(reinterpret_cast<cudaStream_t>(stream), &cs) != cudaSuccess)
      return NUMARCK_ERR_CUDA;
    if (cs != cudaStreamCaptureStatusNone) return NUMARCK_ERR_INVALID_ARG;
  }
  P.sms = device_sms();
  if (P.sms <= 0) return NUMARCK_ERR_CUDA;
  return launch_compress(P, reinterpret_cast<cudaStream_t>(stream));
}

int numarck_read_header(const void* header_host, numarck_header* out) {
  if (!header_host) return NUMARCK_ERR_INVALID_ARG;
  numarck_header h;
  std::memcpy(&h, header_host, sizeof(h));
  const int rc = check_header(h, nullptr);
  if (rc) return rc;
  if (out) *out = h;
  return NUMARCK_OK;
}

int numarck_blob_size(const void* header_host, size_t* bytes) {
  numarck_header h;
  const int rc = numarck_read_header(header_host, &h);
  if (rc) return rc;
  if (bytes) *bytes = (size_t)h.total_bytes;
  return NUMARCK_OK;
}

int numarck_decompress(const void* blob, const void* header_host, const void* prev, void* out,
                       int64_t n, int32_t* status_dev, numarck_stream_t stream) {
  nmk::NvtxRange nvtx_("numarck_decompress");
  if (n < 0) return NUMARCK_ERR_INVALID_ARG;
  return decode(blob, header_host, prev, 0, n, out, n, status_dev, stream);
}

int numarck_decompress_range(const void* blob, const void* header_host, const void* prev_seg,
                             int64_t start, int64_t count, void* out_seg, int32_t* status_dev,
                             numarck_stream_t stream) {
  nmk::NvtxRange nvtx_("numarck_decompress_range");
  return decode(blob, header_host, prev_seg, start, count, out_seg, -1, status_dev, stream);
}

int numarck_decompress_compress(const void* blob, const void* header_host, const void* prev,
                                void* out, int64_t n, int32_t* status_dev, const void* next_cur,
                                const numarck_params* p, void* next_blob, size_t next_blob_cap,
                                void* ws, size_t ws_bytes, numarck_stream_t stream) {
  nmk::NvtxRange nvtx_("numarck_decompress_compress");
  if (n < 0) return NUMARCK_ERR_INVALID_ARG;
  int rc = plan_decompress_check(blob, prev, out, n);
  if (rc) return rc;
  CompressPlan P;
  rc = plan_compress(out, next_cur, n, p, next_blob, next_blob_cap, ws, ws_bytes, &P);
  if (rc) return rc;
  int64_t ntiles = 0;
  if (header_host) {
    numarck_header h;
    std::memcpy(&h, header_host, sizeof(h));
    Geometry g;
    rc = check_header(h, &g);
    if (rc) return rc;
    if (h.n != n || h.dtype != p->dtype) return NUMARCK_ERR_INVALID_ARG;
    ntiles = g.nsub;
  }
  const size_t L = p->dtype == NUMARCK_F64 ? 8 : 4;
  auto overlap = [](const void* a, size_t na, const void* b, size_t nb) {
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return na && nb && x < y + nb && y < x + na;
  };
  const size_t nb = (size_t)n * L;
  if (blob == next_blob || overlap(out, nb, prev, nb) || overlap(out, nb, next_cur, nb) ||
      overlap(out, nb, next_blob, next_blob_cap) || overlap(out, nb, ws, ws_bytes) ||
      overlap(out, nb, blob, NUMARCK_HEADER_BYTES))
    return NUMARCK_ERR_INVALID_ARG;
  if (P.auto_b) {   // as numarck_compress: choosing B synchronises, not allowed while capturing
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(reinterpret_cast<cudaStream_t>(stream), &cs) != cudaSuccess)
      return NUMARCK_ERR_CUDA;
    if (cs != cudaStreamCaptureStatusNone) return NUMARCK_ERR_INVALID_ARG;
  }
  P.sms = device_sms();
  if (P.sms <= 0) return NUMARCK_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n == 0) return launch_compress(P, s);
  DecodePlan D{};
  D.blob = static_cast<const unsigned char*>(blob);
  D.prev_seg = prev;
  D.out_seg = out;
  D.status = status_dev;
  D.start = 0;
  D.count = n;
  D.n_expected = n;
  D.ntiles_hint = ntiles;
  D.sms = P.sms;
  D.status2 = &reinterpret_cast<Ctrl*>(P.ws + P.wl.ctrl)->error;
  D.dtype = p->dtype;
  if (p->anchor == NUMARCK_ANCHOR_MIN) {
    if (launch_decode(D, s) != cudaSuccess) return NUMARCK_ERR_CUDA;
    return launch_compress(P, s);
  }
  trace(0, 6, s);
  if (launch_step(D, P, s) != cudaSuccess) return NUMARCK_ERR_CUDA;
  return launch_compress_tail(P, s);
}

int numarck_selftest_wait(const void* flag_dev, int64_t limit_ns, int32_t* status_dev,
                          numarck_stream_t stream) {
  if (!flag_dev || !status_dev || !aligned(flag_dev, 8) || !aligned(status_dev, 4))
    return NUMARCK_ERR_INVALID_ARG;
  if (limit_ns < 1000000 || limit_ns > 10000000000LL) return NUMARCK_ERR_INVALID_ARG;
  if (launch_wait_selftest(static_cast<const unsigned long long*>(flag_dev),
                           (unsigned long long)limit_ns, status_dev,
                           reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
    return NUMARCK_ERR_CUDA;
  return NUMARCK_OK;
}

int numarck_trace_events(void* const* events, int count) {
  if (count < 0) return NUMARCK_ERR_INVALID_ARG;
  g_trace = count ? events : nullptr;
  g_trace_count = events ? count : 0;
  return NUMARCK_OK;
}

namespace {

int blob_geometry(const void* header_host, Geometry* g) {
  if (!header_host) return NUMARCK_ERR_INVALID_ARG;
  numarck_header h;
  std::memcpy(&h, header_host, sizeof(h));
  return check_header(h, g);
}

}  // namespace

size_t numarck_zindex_bound(const void* header_host) {
  Geometry g;
  if (blob_geometry(header_host, &g)) return 0;
  return (size_t)zindex_bound(g);
}

size_t numarck_zindex_workspace_bytes(const void* header_host) {
  Geometry g;
  if (blob_geometry(header_host, &g)) return 0;
  return (size_t)zindex_workspace(g);
}

int numarck_deflate_index(const void* blob, const void* header_host, void* zindex, size_t zcap,
                          void* ws, size_t ws_bytes, numarck_stream_t stream) {
  nmk::NvtxRange nvtx_("numarck_deflate_index");
  Geometry g;
  int rc = blob_geometry(header_host, &g);
  if (rc) return rc;
  if (!blob || !zindex || !ws || !aligned(blob, 256) || !aligned(zindex, 256) || !aligned(ws, 16))
    return NUMARCK_ERR_INVALID_ARG;
  if (zcap < (size_t)zindex_bound(g) || ws_bytes < (size_t)zindex_workspace(g))
    return NUMARCK_ERR_CAPACITY;
  const int sms = device_sms();
  if (sms <= 0) return NUMARCK_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (g.nsub == 0) {   // no index: the container is its header and one zoff entry
    numarck_zindex_header zh;
    zindex_layout(g, &zh);
    static thread_local unsigned char img[NUMARCK_ZINDEX_HEADER_BYTES + 16];
    std::memcpy(img, &zh, NUMARCK_ZINDEX_HEADER_BYTES);
    const int64_t total = zh.off_data;
    std::memcpy(img + NUMARCK_ZINDEX_HEADER_BYTES, &total, 8);
    if (cudaMemcpyAsync(zindex, img, NUMARCK_ZINDEX_HEADER_BYTES + 8, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return NUMARCK_ERR_CUDA;
    return NUMARCK_OK;
  }
  if (launch_deflate(static_cast<const unsigned char*>(blob), g,
                     static_cast<unsigned char*>(zindex), static_cast<unsigned char*>(ws), sms,
                     s) != cudaSuccess)
    return NUMARCK_ERR_CUDA;
  return NUMARCK_OK;
}

int numarck_inflate_index(const void* zindex, size_t zbytes, const void* header_host, void* blob,
                          int64_t start, int64_t count, int32_t* status_dev,
                          numarck_stream_t stream) {
  nmk::NvtxRange nvtx_("numarck_inflate_index");
  Geometry g;
  int rc = blob_geometry(header_host, &g);
  if (rc) return rc;
  if (!zindex || !blob || !aligned(zindex, 256) || !aligned(blob, 256))
    return NUMARCK_ERR_INVALID_ARG;
  if (start < 0 || count < 0 || start > g.n || count > g.n - start) return NUMARCK_ERR_RANGE;
  if (count == 0) return NUMARCK_OK;
  const int64_t first = start, last = start + count - 1;
  const int64_t q0 = first / g.epb, q1 = last / g.epb;
  const int64_t g0 = q0 * g.spb + (first - q0 * g.epb) / SUB;
  const int64_t g1 = q1 * g.spb + (last - q1 * g.epb) / SUB;
  if (launch_inflate(static_cast<const unsigned char*>(zindex), (long long)zbytes,
                     static_cast<unsigned char*>(blob), g, g0, g1, status_dev,
                     reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
    return NUMARCK_ERR_CUDA;
  return NUMARCK_OK;
}

const char* numarck_status_string(int code) {
  switch (code) {
    case NUMARCK_OK: return "ok";
    case NUMARCK_ERR_INVALID_ARG: return "invalid argument";
    case NUMARCK_ERR_CAPACITY: return "buffer too small";
    case NUMARCK_ERR_CUDA: return "CUDA error";
    case NUMARCK_ERR_CORRUPT: return "corrupt or inconsistent blob";
    case NUMARCK_ERR_RANGE: return "range outside [0, n]";
    case NUMARCK_ERR_TIMEOUT: return "device wait timed out";
    case NUMARCK_ERR_NOMEM: return "out of host memory";
    default: return "unknown status";
  }
}

const char* numarck_version(void) { return "numarck-gb300 1 sm_103a"; }

}  // extern "C"
