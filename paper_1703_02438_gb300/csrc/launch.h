// launch.h — host-side launchers of the NUMARCK kernels (one translation unit per kernel family).
#pragma once

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace nmk {

// An NVTX range around one entry point (header-only NVTX 3: free unless a profiler is attached),
// so that traces group each call's kernels under its name.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Everything a compression launch needs; built and validated by the C ABI (capi.cu).
struct CompressPlan {
  const void* prev;
  const void* cur;
  unsigned char* blob;
  unsigned char* ws;
  WsLayout wl;
  Geometry g;
  numarck_header hdr;      // header as known before the kernels run (n_sel, a, n_inc patched)
  Consts<float> cf;        // valid when dtype == F32
  Consts<double> cd;       // valid when dtype == F64
  bool aligned16;          // prev and cur both 16-byte aligned
  int sms;                 // multiprocessors of the current device
  int64_t code_off;        // byte offset of K1's per-point codes in the blob buffer
  bool auto_b;             // B = 0: choose B from the histogram (§IV.B.2) after K1
};

// Decompression of elements [start, start+count). The kernel takes the blob's geometry from the
// header in device memory and validates it there; n_expected >= 0 must equal the header's n.
// ntiles_hint > 0 (known when the caller supplied a host copy of the header) sizes the grid.
struct DecodePlan {
  const unsigned char* blob;
  const void* prev_seg;
  void* out_seg;
  int32_t* status;
  int64_t start, count, n_expected;
  int64_t ntiles_hint;
  int sms;
  int* status2;            // optional second error word (the next compression's Ctrl::error)
  int dtype;               // element type the blob must hold (0: either)
  int concurrency;         // decodes expected to share the GPU with this one (0 or 1: none)
};

// ---- the fused batch (K6): every phase of the compression of all variables of a batch as one
// persistent launch over a device-side work list, instead of one launch per variable ----

// One variable of a fused batch as the fused kernels read it (device memory, written by the
// upload kernel from the host plan). Its workspace slice has the single-variable layout wl.
struct FusedVar {
  const void* prev;
  const void* cur;
  unsigned char* blob;
  unsigned char* ws;
  Geometry g;
  WsLayout wl;
  double E;
  int64_t block_bytes;
  int64_t code_off;
  int aligned16;
  int pad;
  Consts<double> cd;       // valid when g.dtype == F64
  Consts<float> cf;        // valid when g.dtype == F32
};

// Work-list prefix tables of a fused batch (device memory, count + 1 entries each): the first
// K1 work byte, the first 4096-element tile and the first offset-scan block of each variable.
struct FusedArgs {
  const FusedVar* vars;
  const long long* wpre;
  const long long* tpre;
  const long long* spre;
  unsigned int* ticket;    // offset-scan block order (reset by the upload)
  int count;
  int any_min;             // some variable uses the MIN grid (K0 runs)
  long long WT, NT, NS;    // totals of the three tables
  int exact_warps;         // K3c warps per CTA (4 or 8)
};

// One blob of a fused decode: what the prep kernel validates and the decode kernel reads.
struct FusedDecodeVar {
  const unsigned char* blob;
  const void* prev;
  void* out;
  long long n;
};

struct FusedDecodeArgs {
  const FusedDecodeVar* vars;
  long long* tpre;         // written by the prep kernel: first tile of each blob (count + 1)
  unsigned long long* ticket;   // chunk counter of the decode kernel (reset by the prep kernel)
  int32_t* status;
  int count;
  int seg_log2;            // each tile is decoded by 2^seg_log2 warps
};

cudaError_t launch_fused_hist(const FusedArgs& F, int k1_threads, int sms, cudaStream_t s);
cudaError_t launch_fused_topk(const FusedArgs& F, cudaStream_t s);
cudaError_t launch_fused_assign(const FusedArgs& F, int sms, cudaStream_t s);
cudaError_t launch_fused_offsets(const FusedArgs& F, cudaStream_t s);
cudaError_t launch_fused_exact(const FusedArgs& F, int sms, cudaStream_t s);
cudaError_t launch_fused_decode(const FusedDecodeArgs& D, int sms, cudaStream_t s);

cudaError_t launch_anchor_min(const CompressPlan& P, cudaStream_t s);  // K0 (ANCHOR_MIN only)
cudaError_t launch_hist(const CompressPlan& P, cudaStream_t s);        // K1
cudaError_t launch_auto_b(const CompressPlan& P, cudaStream_t s);      // B from the histogram
// Lossless index compression (k_zlib.cu): container layout and bound for a blob's geometry,
// deflate of every index block, inflate of sub-blocks [g0, g1].
int zindex_layout(const Geometry& g, numarck_zindex_header* zh);
int64_t zindex_bound(const Geometry& g);
int64_t zindex_workspace(const Geometry& g);   // device workspace bytes of launch_deflate
cudaError_t launch_deflate(const unsigned char* blob, const Geometry& g, unsigned char* z,
                           unsigned char* ws, int sms, cudaStream_t s);
cudaError_t launch_inflate(const unsigned char* z, long long zbytes, unsigned char* blob,
                           const Geometry& g, long long g0, long long g1, int32_t* status,
                           cudaStream_t s);
cudaError_t launch_topk(const CompressPlan& P, cudaStream_t s);        // K2
cudaError_t launch_assign(const CompressPlan& P, cudaStream_t s);      // K3a: indices + packing
cudaError_t launch_offsets(const CompressPlan& P, cudaStream_t s);     // K3b: offset tables
cudaError_t launch_exact(const CompressPlan& P, cudaStream_t s);       // K3c: incompressible values
cudaError_t launch_decode(const DecodePlan& P, cudaStream_t s);        // K4 / K5
// one thread running the bounded device wait on a caller's flag (numarck_selftest_wait)
cudaError_t launch_wait_selftest(const unsigned long long* flag, unsigned long long limit_ns,
                                 int32_t* status, cudaStream_t s);
// K41: decompression of D fused with K1 of the compression P of a new timestep against D's
// output (zero-centred grid only)
cudaError_t launch_step(const DecodePlan& D, const CompressPlan& P, cudaStream_t s);

// Host-side planning shared by the single-variable and batched entry points (capi.cu).
int plan_compress(const void* prev, const void* cur, int64_t n, const numarck_params* p,
                  void* blob, size_t blob_cap, void* ws, size_t ws_bytes, CompressPlan* out);
int launch_compress(const CompressPlan& P, cudaStream_t s);
int launch_compress_tail(const CompressPlan& P, cudaStream_t s);   // everything after K1
int plan_decompress_check(const void* blob, const void* prev, void* out, int64_t n);
int launch_decompress(const void* blob, const void* prev, void* out, int64_t n, int32_t* status,
                      int sms, cudaStream_t s, int concurrency = 1);
int current_device_sms();
// Records events[i] of the caller's numarck_trace_events array on s (if set and count >= need).
void trace_event(int i, int need, cudaStream_t s);

}  // namespace nmk
