// batch.cu — compression and decompression of many variables in one call.
//
// The paper stores several compressed variables per file (§IV.D); scientific checkpoints hold
// many variables of very different sizes and types. A batch runs every variable's kernels with
// `lanes` of them in flight at once: variables are assigned to lanes longest-first (the lane
// with the least work so far takes the next largest variable), each lane is a CUDA stream forked
// from the caller's stream with an event and joined back into it, and each lane owns one slice
// of the workspace. Kernel grids of a batch are sized for 1/grid_share of the GPU so that
// several variables share the SMs. The fork/join is made of event records and waits only, so a
// whole batch can be captured into one CUDA graph and replayed.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "launch.h"

using namespace nmk;

namespace {

constexpr int kMaxLanes = 64;
constexpr int kMaxDevices = 64;

struct LanePool {
  bool ready = false;
  cudaStream_t streams[kMaxLanes];
  cudaEvent_t fork;
  cudaEvent_t join[kMaxLanes];
};

std::mutex g_pool_mu;
LanePool g_pools[kMaxDevices];

// Streams and events of the current device (created on first use; kept until process exit).
int lane_pool(LanePool** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NUMARCK_ERR_CUDA;
  LanePool& P = g_pools[dev];
  if (!P.ready) {
    for (int i = 0; i < kMaxLanes; ++i) {
      if (cudaStreamCreateWithFlags(&P.streams[i], cudaStreamNonBlocking) != cudaSuccess)
        return NUMARCK_ERR_CUDA;
      if (cudaEventCreateWithFlags(&P.join[i], cudaEventDisableTiming) != cudaSuccess)
        return NUMARCK_ERR_CUDA;
    }
    if (cudaEventCreateWithFlags(&P.fork, cudaEventDisableTiming) != cudaSuccess)
      return NUMARCK_ERR_CUDA;
    P.ready = true;
  }
  *out = &P;
  return NUMARCK_OK;
}

size_t item_bytes(int64_t n, int dtype) { return (size_t)n * (dtype == NUMARCK_F64 ? 8 : 4); }

// Longest-first assignment of items to lanes (deterministic: ties by index, lanes by index).
std::vector<int> assign_lanes(const int64_t* n, const int* dtype, int count, int lanes) {
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return item_bytes(n[a], dtype[a]) > item_bytes(n[b], dtype[b]);
  });
  std::vector<size_t> load(lanes, 0);
  std::vector<int> lane_of(count, 0);
  for (int i : order) {
    int best = 0;
    for (int l = 1; l < lanes; ++l)
      if (load[l] < load[best]) best = l;
    lane_of[i] = best;
    load[best] += item_bytes(n[i], dtype[i]) + 1;
  }
  return lane_of;
}

int clamp_lanes(int lanes, int count) {
  if (lanes < 1) return 0;
  return std::max(1, std::min({lanes, count, kMaxLanes}));
}

// Workspace slices: slice l is the largest workspace any item of lane l needs, 256-aligned.
int slices(const numarck_batch_item* items, int count, int lanes, std::vector<int>* lane_of,
           std::vector<size_t>* off, size_t* total) {
  std::vector<int64_t> n(count);
  std::vector<int> dt(count);
  for (int i = 0; i < count; ++i) {
    n[i] = items[i].n;
    dt[i] = items[i].params.dtype;
  }
  *lane_of = assign_lanes(n.data(), dt.data(), count, lanes);
  std::vector<size_t> need(lanes, 0);
  for (int i = 0; i < count; ++i) {
    if (items[i].params.B == 0) return NUMARCK_ERR_INVALID_ARG;   // automatic B synchronises
    const size_t w = numarck_workspace_bytes(items[i].n, &items[i].params);
    if (w == 0) return NUMARCK_ERR_INVALID_ARG;
    need[(*lane_of)[i]] = std::max(need[(*lane_of)[i]], w);
  }
  off->assign(lanes, 0);
  size_t o = 0;
  for (int l = 0; l < lanes; ++l) {
    (*off)[l] = o;
    o += (need[l] + 255) / 256 * 256;
  }
  *total = o;
  return NUMARCK_OK;
}

}  // namespace

extern "C" {

size_t numarck_batch_workspace_bytes(const numarck_batch_item* items, int count, int lanes) {
  if (!items || count <= 0) return 0;
  lanes = clamp_lanes(lanes, count);
  if (lanes == 0) return 0;
  std::vector<int> lane_of;
  std::vector<size_t> off;
  size_t total = 0;
  if (slices(items, count, lanes, &lane_of, &off, &total)) return 0;
  return total;
}

int numarck_compress_batch(const numarck_batch_item* items, int count, int lanes, int grid_share,
                           void* ws, size_t ws_bytes, numarck_stream_t stream) {
  nmk::NvtxRange nvtx_("numarck_compress_batch");
  if (!items || count < 0 || grid_share < 1) return NUMARCK_ERR_INVALID_ARG;
  if (count == 0) return NUMARCK_OK;
  lanes = clamp_lanes(lanes, count);
  if (lanes == 0) return NUMARCK_ERR_INVALID_ARG;
  std::vector<int> lane_of;
  std::vector<size_t> off;
  size_t total = 0;
  int rc = slices(items, count, lanes, &lane_of, &off, &total);
  if (rc) return rc;
  if (!ws) return NUMARCK_ERR_INVALID_ARG;
  if (ws_bytes < total) return NUMARCK_ERR_CAPACITY;
  // validate and plan every item before launching anything
  std::vector<CompressPlan> plans(count);
  unsigned char* base = static_cast<unsigned char*>(ws);
  for (int i = 0; i < count; ++i) {
    const numarck_batch_item& it = items[i];
    const size_t slice = (lane_of[i] + 1 < lanes ? off[lane_of[i] + 1] : total) - off[lane_of[i]];
    rc = plan_compress(it.prev, it.cur, it.n, &it.params, it.blob, it.blob_cap,
                       base + off[lane_of[i]], slice, &plans[i]);
    if (rc) return rc;
  }
  const int sms = current_device_sms();
  if (sms <= 0) return NUMARCK_ERR_CUDA;
  const int share_sms = std::max(1, sms / grid_share);
  std::lock_guard<std::mutex> lock(g_pool_mu);
  LanePool* P = nullptr;
  if ((rc = lane_pool(&P))) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaEventRecord(P->fork, s) != cudaSuccess) return NUMARCK_ERR_CUDA;
  for (int l = 0; l < lanes; ++l)
    if (cudaStreamWaitEvent(P->streams[l], P->fork, 0) != cudaSuccess) return NUMARCK_ERR_CUDA;
  for (int i = 0; i < count; ++i) {
    plans[i].sms = share_sms;
    if ((rc = launch_compress(plans[i], P->streams[lane_of[i]]))) return rc;
  }
  for (int l = 0; l < lanes; ++l) {
    if (cudaEventRecord(P->join[l], P->streams[l]) != cudaSuccess) return NUMARCK_ERR_CUDA;
    if (cudaStreamWaitEvent(s, P->join[l], 0) != cudaSuccess) return NUMARCK_ERR_CUDA;
  }
  return NUMARCK_OK;
}

int numarck_decompress_batch(const numarck_batch_decode_item* items, int count, int lanes,
                             int grid_share, int32_t* status_dev, numarck_stream_t stream) {
  nmk::NvtxRange nvtx_("numarck_decompress_batch");
  if (!items || count < 0 || grid_share < 1) return NUMARCK_ERR_INVALID_ARG;
  if (count == 0) return NUMARCK_OK;
  lanes = clamp_lanes(lanes, count);
  if (lanes == 0) return NUMARCK_ERR_INVALID_ARG;
  std::vector<int64_t> n(count);
  std::vector<int> dt(count, NUMARCK_F64);
  for (int i = 0; i < count; ++i) {
    int rc = plan_decompress_check(items[i].blob, items[i].prev, items[i].out, items[i].n);
    if (rc) return rc;
    n[i] = items[i].n;
  }
  const std::vector<int> lane_of = assign_lanes(n.data(), dt.data(), count, lanes);
  const int sms = current_device_sms();
  if (sms <= 0) return NUMARCK_ERR_CUDA;
  const int share_sms = std::max(1, sms / grid_share);
  std::lock_guard<std::mutex> lock(g_pool_mu);
  LanePool* P = nullptr;
  int rc = lane_pool(&P);
  if (rc) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaEventRecord(P->fork, s) != cudaSuccess) return NUMARCK_ERR_CUDA;
  for (int l = 0; l < lanes; ++l)
    if (cudaStreamWaitEvent(P->streams[l], P->fork, 0) != cudaSuccess) return NUMARCK_ERR_CUDA;
  for (int i = 0; i < count; ++i)
    if ((rc = launch_decompress(items[i].blob, items[i].prev, items[i].out, items[i].n,
                                status_dev, share_sms, P->streams[lane_of[i]],
                                std::max(1, lanes / grid_share))))
      return rc;
  for (int l = 0; l < lanes; ++l) {
    if (cudaEventRecord(P->join[l], P->streams[l]) != cudaSuccess) return NUMARCK_ERR_CUDA;
    if (cudaStreamWaitEvent(s, P->join[l], 0) != cudaSuccess) return NUMARCK_ERR_CUDA;
  }
  return NUMARCK_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// The fused batch (K6): each phase of the compression (K0/K1, K2, K3a + K3f, K3b, K3c) of every
// variable runs as ONE persistent launch over a device-side work list (variables' bytes, tiles
// and scan blocks, concatenated), with each item's dtype, E and B read from the variable's
// descriptor; the decompression likewise (one prep launch, one decode launch). The descriptors
// and prefix tables are written into the workspace by upload kernels whose parameters carry
// them, so a call is a fixed sequence of kernel launches that a CUDA graph can capture.
// ---------------------------------------------------------------------------------------
namespace {

constexpr int kUploadVars = 64;            // descriptors per upload launch (parameter space)
constexpr int kUploadWords = 3800;         // int64 prefix entries per upload launch
constexpr int kUploadDecode = 512;
constexpr int kMaxGroups = 64;

struct UploadVars {
  FusedVar v[kUploadVars];
  int first, n;
  int groups;                               // tickets to reset (with the first chunk)
};
static_assert(sizeof(UploadVars) <= 32000, "upload chunk must fit the kernel parameter space");

struct UploadWords {
  long long w[kUploadWords];
  int first, n;
};
static_assert(sizeof(UploadWords) <= 32000, "upload chunk must fit the kernel parameter space");

struct UploadDecodeChunk {
  FusedDecodeVar v[kUploadDecode];
  int first, n;
};
static_assert(sizeof(UploadDecodeChunk) <= 32000, "upload chunk must fit the kernel parameter space");

__global__ void k_fused_upload_vars(UploadVars C, FusedVar* vars, unsigned int* tickets) {
  const int i = (int)threadIdx.x;
  if (i < C.n) vars[C.first + i] = C.v[i];
  if (C.first == 0 && i < C.groups) tickets[i] = 0u;
}

__global__ void k_fused_upload_words(UploadWords C, long long* words) {
  for (int i = (int)threadIdx.x; i < C.n; i += blockDim.x) words[C.first + i] = C.w[i];
}

__global__ void k_fused_upload_decode(UploadDecodeChunk C, FusedDecodeVar* vars) {
  for (int i = (int)threadIdx.x; i < C.n; i += blockDim.x) vars[C.first + i] = C.v[i];
}

// Workspace of a fused compression: a 256-byte control block (one offset-scan ticket per group),
// the variable descriptors (grouped), the three prefix tables of every group (count + groups
// entries each), then one single-variable workspace slice per variable (in item order).
struct FusedLayout {
  size_t vars, pre, slices, total;
  std::vector<size_t> slice;                // offset of variable v's slice
};

size_t r256(size_t x) { return (x + 255) / 256 * 256; }

int fused_layout(const numarck_batch_item* items, int count, FusedLayout* L) {
  if (!items || count <= 0) return NUMARCK_ERR_INVALID_ARG;
  size_t o = 256;
  L->vars = o;
  o = r256(o + sizeof(FusedVar) * (size_t)count);
  L->pre = o;
  o = r256(o + 3 * 8 * (size_t)(count + kMaxGroups));
  L->slices = o;
  L->slice.assign(count, 0);
  for (int i = 0; i < count; ++i) {
    if (items[i].params.B == 0) return NUMARCK_ERR_INVALID_ARG;   // automatic B synchronises
    const size_t w = numarck_workspace_bytes(items[i].n, &items[i].params);
    if (w == 0) return NUMARCK_ERR_INVALID_ARG;
    L->slice[i] = o;
    o = r256(o + w);
  }
  L->total = o;
  return NUMARCK_OK;
}

int check_tuning(const numarck_fused_tuning* t, numarck_fused_tuning* out) {
  numarck_fused_tuning d{1024, 8, 0, 1, 1, 0};
  if (t) {
    if (t->reserved != 0) return NUMARCK_ERR_INVALID_ARG;
    if (t->k1_threads) d.k1_threads = t->k1_threads;
    if (t->exact_warps) d.exact_warps = t->exact_warps;
    d.decode_seg_log2 = t->decode_seg_log2;
    if (t->groups) d.groups = t->groups;
    if (t->streams) d.streams = t->streams;
  }
  if (d.k1_threads != 512 && d.k1_threads != 1024) return NUMARCK_ERR_INVALID_ARG;
  if (d.exact_warps != 4 && d.exact_warps != 8) return NUMARCK_ERR_INVALID_ARG;
  if (d.decode_seg_log2 < 0 || d.decode_seg_log2 > 3) return NUMARCK_ERR_INVALID_ARG;
  if (d.groups < 1 || d.groups > kMaxGroups) return NUMARCK_ERR_INVALID_ARG;
  if (d.streams < 1 || d.streams > 8) return NUMARCK_ERR_INVALID_ARG;
  *out = d;
  return NUMARCK_OK;
}

// The fused launches of one group on stream s (its grids sized for `sms` multiprocessors).
int run_fused_group(const FusedArgs& F, const numarck_fused_tuning& tu, int sms, cudaStream_t s,
                    bool trace) {
  if (launch_fused_hist(F, tu.k1_threads, sms, s) != cudaSuccess) return NUMARCK_ERR_CUDA;
  if (trace) trace_event(1, 6, s);
  if (launch_fused_topk(F, s) != cudaSuccess) return NUMARCK_ERR_CUDA;
  if (trace) trace_event(2, 6, s);
  if (launch_fused_assign(F, sms, s) != cudaSuccess) return NUMARCK_ERR_CUDA;
  if (trace) trace_event(3, 6, s);
  if (launch_fused_offsets(F, s) != cudaSuccess) return NUMARCK_ERR_CUDA;
  if (trace) trace_event(4, 6, s);
  if (launch_fused_exact(F, sms, s) != cudaSuccess) return NUMARCK_ERR_CUDA;
  if (trace) trace_event(5, 6, s);
  return NUMARCK_OK;
}

}  // namespace

extern "C" {

size_t numarck_fused_workspace_bytes(const numarck_batch_item* items, int count) {
  FusedLayout L;
  if (fused_layout(items, count, &L)) return 0;
  return L.total;
}

int numarck_compress_batch_fused(const numarck_batch_item* items, int count,
                                 const numarck_fused_tuning* tuning, void* ws, size_t ws_bytes,
                                 numarck_stream_t stream) {
  nmk::NvtxRange nvtx_("numarck_compress_batch_fused");
  if (!items || count < 0) return NUMARCK_ERR_INVALID_ARG;
  if (count == 0) return NUMARCK_OK;
  numarck_fused_tuning tu;
  int rc = check_tuning(tuning, &tu);
  if (rc) return rc;
  FusedLayout L;
  if ((rc = fused_layout(items, count, &L))) return rc;
  if (!ws || ((uintptr_t)ws % 256)) return NUMARCK_ERR_INVALID_ARG;
  if (ws_bytes < L.total) return NUMARCK_ERR_CAPACITY;
  unsigned char* base = static_cast<unsigned char*>(ws);
  // validate and plan every variable before launching anything
  std::vector<FusedVar> plan(count);
  int any_min = 0;
  for (int i = 0; i < count; ++i) {
    const numarck_batch_item& it = items[i];
    const size_t slice = (i + 1 < count ? L.slice[i + 1] : L.total) - L.slice[i];
    CompressPlan P;
    if ((rc = plan_compress(it.prev, it.cur, it.n, &it.params, it.blob, it.blob_cap,
                            base + L.slice[i], slice, &P)))
      return rc;
    FusedVar& V = plan[i];
    std::memset(&V, 0, sizeof(V));
    V.prev = it.prev;
    V.cur = it.cur;
    V.blob = P.blob;
    V.ws = P.ws;
    V.g = P.g;
    V.wl = P.wl;
    V.E = it.params.E;
    V.block_bytes = P.hdr.block_bytes;
    V.code_off = P.code_off;
    V.aligned16 = P.aligned16 ? 1 : 0;
    V.cd = P.cd;
    V.cf = P.cf;
    any_min |= P.g.anchor == NUMARCK_ANCHOR_MIN;
  }
  const int groups = std::min(tu.groups, count);
  const int streams = std::min(tu.streams, groups);
  // groups of about equal bytes (longest first), each in item order; descriptors group-major
  std::vector<int64_t> nn(count);
  std::vector<int> dt(count);
  for (int i = 0; i < count; ++i) {
    nn[i] = items[i].n;
    dt[i] = items[i].params.dtype;
  }
  const std::vector<int> group_of = assign_lanes(nn.data(), dt.data(), count, groups);
  std::vector<FusedVar> vars;
  vars.reserve(count);
  std::vector<long long> pre(3 * (size_t)(count + kMaxGroups), 0);
  const size_t stride = (size_t)(count + kMaxGroups);   // table t of all groups at t * stride
  std::vector<FusedArgs> F(groups);
  for (int g = 0; g < groups; ++g) {
    const int v0 = (int)vars.size();
    const size_t p0 = (size_t)v0 + g;       // the group's first prefix entry
    long long w = 0, t = 0, sb = 0;
    for (int i = 0; i < count; ++i) {
      if (group_of[i] != g) continue;
      const FusedVar& V = plan[i];
      const size_t k = p0 + (vars.size() - v0);
      pre[k] = w;
      pre[stride + k] = t;
      pre[2 * stride + k] = sb;
      w += V.g.n * (V.g.dtype == NUMARCK_F64 ? 8 : 4);
      t += V.g.nsub;
      sb += (V.g.nsub + SCAN_TILE - 1) / SCAN_TILE;
      vars.push_back(V);
    }
    const int cnt = (int)vars.size() - v0;
    pre[p0 + cnt] = w;
    pre[stride + p0 + cnt] = t;
    pre[2 * stride + p0 + cnt] = sb;
    FusedArgs& A = F[g];
    A = FusedArgs{};
    A.vars = reinterpret_cast<const FusedVar*>(base + L.vars) + v0;
    A.wpre = reinterpret_cast<const long long*>(base + L.pre) + p0;
    A.tpre = reinterpret_cast<const long long*>(base + L.pre) + stride + p0;
    A.spre = reinterpret_cast<const long long*>(base + L.pre) + 2 * stride + p0;
    A.ticket = reinterpret_cast<unsigned int*>(base) + g;
    A.count = cnt;
    A.any_min = any_min;
    A.WT = w;
    A.NT = t;
    A.NS = sb;
    A.exact_warps = tu.exact_warps;
  }
  const int sms = current_device_sms();
  if (sms <= 0) return NUMARCK_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  trace_event(0, 6, s);
  for (int first = 0; first < count; first += kUploadVars) {
    UploadVars C;
    std::memset(&C, 0, sizeof(C));
    C.first = first;
    C.n = std::min(kUploadVars, count - first);
    C.groups = groups;
    for (int i = 0; i < C.n; ++i) C.v[i] = vars[first + i];
    k_fused_upload_vars<<<1, kUploadVars, 0, s>>>(
        C, reinterpret_cast<FusedVar*>(base + L.vars), reinterpret_cast<unsigned int*>(base));
    if (cudaGetLastError() != cudaSuccess) return NUMARCK_ERR_CUDA;
  }
  for (size_t first = 0; first < pre.size(); first += kUploadWords) {
    UploadWords C;
    C.first = (int)first;
    C.n = (int)std::min<size_t>(kUploadWords, pre.size() - first);
    std::memcpy(C.w, pre.data() + first, sizeof(long long) * C.n);
    k_fused_upload_words<<<1, 256, 0, s>>>(C, reinterpret_cast<long long*>(base + L.pre));
    if (cudaGetLastError() != cudaSuccess) return NUMARCK_ERR_CUDA;
  }
  if (streams == 1) {
    for (int g = 0; g < groups; ++g)
      if ((rc = run_fused_group(F[g], tu, sms, s, groups == 1))) return rc;
    if (groups > 1) trace_event(5, 6, s);
    return NUMARCK_OK;
  }
  // groups round-robin on the library's lane streams, forked from and joined into `stream`
  std::lock_guard<std::mutex> lock(g_pool_mu);
  LanePool* LP = nullptr;
  if ((rc = lane_pool(&LP))) return rc;
  if (cudaEventRecord(LP->fork, s) != cudaSuccess) return NUMARCK_ERR_CUDA;
  for (int l = 0; l < streams; ++l)
    if (cudaStreamWaitEvent(LP->streams[l], LP->fork, 0) != cudaSuccess) return NUMARCK_ERR_CUDA;
  const int share = std::max(1, sms / streams);
  for (int g = 0; g < groups; ++g)
    if ((rc = run_fused_group(F[g], tu, share, LP->streams[g % streams], false))) return rc;
  for (int l = 0; l < streams; ++l) {
    if (cudaEventRecord(LP->join[l], LP->streams[l]) != cudaSuccess) return NUMARCK_ERR_CUDA;
    if (cudaStreamWaitEvent(s, LP->join[l], 0) != cudaSuccess) return NUMARCK_ERR_CUDA;
  }
  trace_event(5, 6, s);
  return NUMARCK_OK;
}

size_t numarck_fused_decode_workspace_bytes(int count) {
  if (count <= 0) return 0;
  return 256 + r256(sizeof(FusedDecodeVar) * (size_t)count) + r256(8 * (size_t)(count + 1));
}

int numarck_decompress_batch_fused(const numarck_batch_decode_item* items, int count,
                                   const numarck_fused_tuning* tuning, void* ws, size_t ws_bytes,
                                   int32_t* status_dev, numarck_stream_t stream) {
  nmk::NvtxRange nvtx_("numarck_decompress_batch_fused");
  if (!items || count < 0) return NUMARCK_ERR_INVALID_ARG;
  if (count == 0) return NUMARCK_OK;
  numarck_fused_tuning tu;
  int rc = check_tuning(tuning, &tu);
  if (rc) return rc;
  if (!ws || ((uintptr_t)ws % 256)) return NUMARCK_ERR_INVALID_ARG;
  if (ws_bytes < numarck_fused_decode_workspace_bytes(count)) return NUMARCK_ERR_CAPACITY;
  for (int i = 0; i < count; ++i)
    if ((rc = plan_decompress_check(items[i].blob, items[i].prev, items[i].out, items[i].n)))
      return rc;
  const int sms = current_device_sms();
  if (sms <= 0) return NUMARCK_ERR_CUDA;
  unsigned char* base = static_cast<unsigned char*>(ws);
  FusedDecodeArgs D{};
  D.ticket = reinterpret_cast<unsigned long long*>(base);
  D.vars = reinterpret_cast<const FusedDecodeVar*>(base + 256);
  D.tpre = reinterpret_cast<long long*>(base + 256 + r256(sizeof(FusedDecodeVar) * (size_t)count));
  D.status = status_dev;
  D.count = count;
  D.seg_log2 = tu.decode_seg_log2;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  trace_event(0, 2, s);
  for (int first = 0; first < count; first += kUploadDecode) {
    UploadDecodeChunk C;
    std::memset(&C, 0, sizeof(C));
    C.first = first;
    C.n = std::min(kUploadDecode, count - first);
    for (int i = 0; i < C.n; ++i) {
      const numarck_batch_decode_item& it = items[first + i];
      C.v[i] = FusedDecodeVar{static_cast<const unsigned char*>(it.blob), it.prev, it.out, it.n};
    }
    k_fused_upload_decode<<<1, 256, 0, s>>>(C, const_cast<FusedDecodeVar*>(D.vars));
    if (cudaGetLastError() != cudaSuccess) return NUMARCK_ERR_CUDA;
  }
  if (launch_fused_decode(D, sms, s) != cudaSuccess) return NUMARCK_ERR_CUDA;
  trace_event(1, 2, s);
  return NUMARCK_OK;
}

}  // extern "C"
