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
