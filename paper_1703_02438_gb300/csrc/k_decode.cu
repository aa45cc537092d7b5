// k_decode.cu — K4/K5: decompression (§III.E, Eq. 4 read as R = prev * (1 + centre)) and
// partial decompression of a segment (§IV.C, §V.C).
//
// One tile = one 4096-element sub-block. A tile loads its packed index bits into shared memory,
// unpacks B-bit fields, numbers its incompressible points in element order (warp ballots and a
// scan over 32-element chunks) and takes their values from the incompressible table starting at
// the sub-block's offset; every other point is prev * m[idx] with m = 1 + centre computed in T
// once per CTA. Tiles are independent, so the kernel is a persistent grid with a static tile
// stride. A segment decode touches only the tiles that overlap it (the paper decodes the index
// blocks that cover the segment and finds its first incompressible value through the per-block
// offset table; the per-sub-block table refines that to 4096 elements).
//
// The kernel reads the blob header from device memory and validates it (magic, version, status
// word, geometry implied by n/B/block size, counts), so decompression needs no host round trip
// after compression: a compress -> decompress chain stays asynchronous on one stream.
#include "launch.h"

namespace nmk {

namespace {

struct DecodeArgs {
  const unsigned char* blob;
  const void* prev_seg;
  void* out_seg;
  int32_t* status;
  long long start, count, n_expected;
};

template <typename T>
struct BitsOf;
template <>
struct BitsOf<float> {
  using U = unsigned int;
};
template <>
struct BitsOf<double> {
  using U = unsigned long long;
};

constexpr int K4_WARPS = 16;                    // warps per CTA (each owns whole tiles)
constexpr int K4_THREADS = K4_WARPS * 32;
constexpr int K4_CHUNK = 1024;                  // elements decoded per step of a warp
constexpr int K4_UNROLL = 8;                    // 32-element steps whose loads are in flight
constexpr int K4_WORDS = K4_CHUNK * NUMARCK_MAX_B / 32 + 8;   // packed words of a chunk (+guard)
constexpr int K4_DYN_SMEM = DM_SMEM * 8 + K4_WARPS * K4_WORDS * 4;

// One warp decodes one 4096-element tile at a time, in 1024-element chunks: it copies the
// chunk's packed bits into its shared buffer, unpacks B-bit fields, and walks the chunk in
// 32-element steps, numbering incompressible points with ballots from the tile's entry in the
// sub-block offset table. No block-wide barrier is needed after the multiplier table is built.
template <typename T>
__device__ __forceinline__ void decode_tiles(const DecodeArgs& A, const Geometry& g,
                                             long long n_inc, long long g0, long long g1,
                                             unsigned char* dyn) {
  const int tid = (int)threadIdx.x;
  const int lane = (int)lane_id();
  const int warp = tid >> 5;
  const int B = g.B;
  const unsigned M = (unsigned)g.M;
  const unsigned mask = (1u << B) - 1u;
  const T* centres = reinterpret_cast<const T*>(A.blob + g.off_centres);
  const int64_t* idx_off = reinterpret_cast<const int64_t*>(A.blob + g.off_idx_off);
  const int64_t* sub_off = reinterpret_cast<const int64_t*>(A.blob + g.off_sub_off);
  using U = typename BitsOf<T>::U;
  const U* exact_u = reinterpret_cast<const U*>(A.blob + g.off_exact);
  const unsigned char* index = A.blob + g.off_index;
  const T* prev = static_cast<const T*>(A.prev_seg);
  T* out = static_cast<T*>(A.out_seg);
  U* out_u = reinterpret_cast<U*>(A.out_seg);
  T* s_m = reinterpret_cast<T*>(dyn);
  unsigned* words = reinterpret_cast<unsigned*>(dyn + DM_SMEM * 8) + warp * K4_WORDS;

  const int nm = min(1 << B, DM_SMEM);
  for (int r = tid; r < nm; r += K4_THREADS) s_m[r] = t_add((T)1, centres[r]);
  __syncthreads();   // the only block-wide barrier

  const long long seg_lo = A.start, seg_hi = A.start + A.count;
  const long long W = (long long)gridDim.x * K4_WARPS;
  for (long long gt = g0 + (long long)blockIdx.x * K4_WARPS + warp; gt <= g1; gt += W) {
    const long long q = gt / g.spb, t = gt - q * g.spb;
    const long long j0 = q * g.epb + t * SUB;
    const long long bend = min((long long)g.n, (long long)((q + 1) * g.epb));
    const int cnt = (int)min((long long)SUB, bend - j0);
    const long long base = sub_off[gt];
    const long long boff = idx_off[q];
    const long long tstart = boff + t * (long long)(SUB / 8 * B);
    const long long tend = tstart + 16LL * (((cnt * B + 7) / 8 + 15) / 16);
    if (base < 0 || base > n_inc || (boff & 15) || boff < 0 || tend > g.index_bytes) {
      if (lane == 0 && A.status) atomicExch(A.status, NUMARCK_ERR_CORRUPT);
      continue;
    }
    long long run = base;
    bool whole = true;
    for (int c0 = 0; c0 < cnt; c0 += K4_CHUNK) {
      const long long cj = j0 + c0;
      if (cj >= seg_hi) { whole = false; break; }
      const int ccnt = min(K4_CHUNK, cnt - c0);
      const int nv16 = (((ccnt * B + 7) >> 3) + 15) >> 4;
      const uint4* src = reinterpret_cast<const uint4*>(index + tstart + (c0 / 8) * B);
      for (int v = lane; v < nv16; v += 32) reinterpret_cast<uint4*>(words)[v] = __ldcs(src + v);
      if (lane < 4) words[nv16 * 4 + lane] = 0u;
      __syncwarp();
      const bool emit = cj + ccnt > seg_lo;   // else: only count this chunk's markers
      for (int i0 = 0; i0 < K4_CHUNK / 32; i0 += K4_UNROLL) {
        T pv[K4_UNROLL];
#pragma unroll
        for (int u = 0; u < K4_UNROLL; ++u) {
          const int e = (i0 + u) * 32 + lane;
          const long long j = cj + e;
          pv[u] = (emit && e < ccnt && j >= seg_lo && j < seg_hi) ? ld_stream(prev + (j - seg_lo))
                                                                   : (T)0;
        }
#pragma unroll
        for (int u = 0; u < K4_UNROLL; ++u) {
          const int e = (i0 + u) * 32 + lane;
          unsigned id = 0;
          if (e < ccnt) {
            const unsigned bp = (unsigned)e * (unsigned)B;
            const unsigned w = bp >> 5, o = bp & 31u;
            const unsigned long long v2 =
                ((unsigned long long)words[w + 1] << 32) | (unsigned long long)words[w];
            id = (unsigned)(v2 >> o) & mask;
          }
          const bool mk = e < ccnt && id == M;
          const unsigned ball = __ballot_sync(0xffffffffu, mk);
          const long long j = cj + e;
          if (emit && e < ccnt && j >= seg_lo && j < seg_hi) {
            const long long o = j - seg_lo;
            if (mk) {
              const long long pos = run + __popc(ball & lanemask_lt());
              if (pos < n_inc) {
                out_u[o] = exact_u[pos];
              } else {
                out_u[o] = 0;
                if (A.status) atomicExch(A.status, NUMARCK_ERR_CORRUPT);
              }
            } else {
              const T m = id < (unsigned)DM_SMEM ? s_m[id] : t_add((T)1, centres[id]);
              out[o] = t_mul(pv[u], m);
            }
          }
          run += __popc(ball);
        }
      }
      __syncwarp();
    }
    if (whole && lane == 0 && A.status) {
      const long long next = (gt + 1 < g.nsub) ? sub_off[gt + 1] : n_inc;
      if (run != next) atomicExch(A.status, NUMARCK_ERR_CORRUPT);
    }
  }
}

__global__ void __launch_bounds__(K4_THREADS, 2) k4_decode(DecodeArgs A) {
  extern __shared__ __align__(16) unsigned char k4_dyn[];
  __shared__ __align__(16) numarck_header s_h;
  __shared__ Geometry s_g;
  __shared__ long long s_g0, s_g1;
  __shared__ int s_ok;
  if (threadIdx.x < NUMARCK_HEADER_BYTES / 16)
    reinterpret_cast<uint4*>(&s_h)[threadIdx.x] = reinterpret_cast<const uint4*>(A.blob)[threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) {
    Geometry g{};
    int rc = check_header(s_h, &g);
    if (!rc && A.n_expected >= 0 && A.n_expected != s_h.n) rc = NUMARCK_ERR_INVALID_ARG;
    if (!rc && (A.start < 0 || A.count < 0 || A.start > s_h.n || A.count > s_h.n - A.start))
      rc = NUMARCK_ERR_RANGE;
    const unsigned L = s_h.dtype == NUMARCK_F64 ? 8u : 4u;
    if (!rc && (((uintptr_t)A.prev_seg | (uintptr_t)A.out_seg) % L)) rc = NUMARCK_ERR_INVALID_ARG;
    long long g0 = 0, g1 = -1;
    if (!rc && A.count > 0) {
      const long long first = A.start, last = A.start + A.count - 1;
      const long long q0 = first / g.epb, q1 = last / g.epb;
      g0 = q0 * g.spb + (first - q0 * g.epb) / SUB;
      g1 = q1 * g.spb + (last - q1 * g.epb) / SUB;
    }
    if (rc && blockIdx.x == 0 && A.status) atomicExch(A.status, rc);
    s_ok = rc == 0 && g1 >= g0 + (long long)blockIdx.x * K4_WARPS;
    s_g = g;
    s_g0 = g0;
    s_g1 = g1;
  }
  __syncthreads();
  if (!s_ok) return;
  const Geometry g = s_g;
  if (g.dtype == NUMARCK_F64)
    decode_tiles<double>(A, g, s_h.n_inc, s_g0, s_g1, k4_dyn);
  else
    decode_tiles<float>(A, g, s_h.n_inc, s_g0, s_g1, k4_dyn);
}

}  // namespace

cudaError_t launch_decode(const DecodePlan& P, cudaStream_t s) {
  if (P.count <= 0) return cudaSuccess;
  static int occ[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  int per_sm = dev < 64 ? occ[dev] : 0;
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k4_decode, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         K4_DYN_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k4_decode, K4_THREADS, K4_DYN_SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (dev < 64) occ[dev] = per_sm;
  }
  long long blocks = (long long)P.sms * per_sm;
  if (P.ntiles_hint > 0) {
    const long long need = (P.ntiles_hint + K4_WARPS - 1) / K4_WARPS;
    if (blocks > need) blocks = need;
  }
  DecodeArgs A{P.blob, P.prev_seg, P.out_seg, P.status, P.start, P.count, P.n_expected};
  k4_decode<<<(int)blocks, K4_THREADS, K4_DYN_SMEM, s>>>(A);
  return cudaGetLastError();
}

}  // namespace nmk
