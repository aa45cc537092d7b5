// k_decode.cu — K4/K5: decompression (§III.E, Eq. 4 read as R = prev * (1 + centre)) and
// partial decompression of a segment (§IV.C, §V.C).
//
// One warp decodes one 4096-element tile (sub-block), or one of 2, 4 or 8 parts of it when a
// variable has too few tiles to fill the GPU (see seg_log2_for), in 128-element steps where lane
// l owns elements 4l .. 4l+3: it reads its 4B-bit field of the step's packed image (one word
// when B = 8, two when B = 16, else the two or three words the field overlaps), splits it into
// four indices, numbers the incompressible points of the step in element order with four
// ballots from the tile's entry in the sub-block offset table, and writes prev * m[idx] or the
// incompressible value; prev and R move as 16-byte vectors when the tile lies inside the
// segment and both pointers are aligned. m = 1 + centre is computed in T once per CTA. Tiles
// are independent, so the kernel is a persistent grid with a static tile stride. A segment
// decode touches only the tiles that overlap it (the paper decodes the index blocks that cover
// the segment and finds its first incompressible value through the per-block offset table; the
// per-sub-block table refines that to 4096 elements). B, read from the header on the device, is
// dispatched once per CTA to a body compiled for that width.
//
// The kernel reads the blob header from device memory and validates it (magic, version, status
// word, geometry implied by n/B/block size, counts), so decompression needs no host round trip
// after compression: a compress -> decompress chain stays asynchronous on one stream.
#include <algorithm>

#include "k4.cuh"

namespace nmk {

namespace {

template <typename T, int B>
__device__ __forceinline__ void decode_tiles(const DecodeArgs& A, const Geometry& g,
                                             long long n_inc, long long g0, long long g1,
                                             const T* s_m) {
  using U = typename BitsOf<T>::U;
  using F = typename Field<B>::type;
  constexpr int FB = 4 * B;
  const int lane = (int)lane_id();
  const int warp = (int)(threadIdx.x >> 5);
  const T* centres = reinterpret_cast<const T*>(A.blob + g.off_centres);
  const int64_t* idx_off = reinterpret_cast<const int64_t*>(A.blob + g.off_idx_off);
  const int64_t* sub_off = reinterpret_cast<const int64_t*>(A.blob + g.off_sub_off);
  const U* exact_u = reinterpret_cast<const U*>(A.blob + g.off_exact);
  const unsigned char* index = A.blob + g.off_index;
  const T* prev = static_cast<const T*>(A.prev_seg);
  T* out = static_cast<T*>(A.out_seg);
  const unsigned lt = lanemask_lt();

  const long long seg_lo = A.start, seg_hi = A.start + A.count;
  const long long W = (long long)gridDim.x * K4_WARPS;
  const int sl = A.seg_log2;                     // units: 2^sl segments per sub-block
  const int seglen = SUB >> sl;
  const long long u1 = (g1 + 1) << sl;
  for (long long u = (g0 << sl) + (long long)blockIdx.x * K4_WARPS + warp; u < u1; u += W) {
    const long long gt = u >> sl;
    const int sbeg = (int)(u & ((1 << sl) - 1)) * seglen;
    const long long q = gt / g.spb, t = gt - q * g.spb;
    const long long j0 = q * g.epb + t * SUB;
    const long long bend = min((long long)g.n, (long long)((q + 1) * g.epb));
    const int cnt = (int)min((long long)SUB, bend - j0);
    const long long base = sub_off[gt];
    const long long boff = idx_off[q];
    const long long tstart = boff + t * (long long)(SUB / 8 * B);
    const int twords = 4 * ((cnt * B + 127) / 128);
    if (base < 0 || base > n_inc || (boff & 15) || boff < 0 ||
        tstart + 4LL * twords > g.index_bytes) {
      if (lane == 0) report(A, NUMARCK_ERR_CORRUPT);
      continue;
    }
    const unsigned* tw = reinterpret_cast<const unsigned*>(index + tstart);
    // elements [e_lo, e_hi) of the tile lie in the requested range; pt/ot address tile element 0
    const int e_lo = (int)max(0LL, seg_lo - j0);
    const int e_hi = (int)min((long long)cnt, seg_hi - j0);
    // this warp's steps: [sbeg, send) of the tile, up to e_hi
    const int send = min(min(cnt, sbeg + seglen), e_hi);
    if (sbeg >= send || sbeg + seglen <= e_lo) continue;
    const T* pt = prev + (j0 - seg_lo);
    T* ot = out + (j0 - seg_lo);
    const bool vec = e_lo == 0 && ((reinterpret_cast<uintptr_t>(pt) |
                                    reinterpret_cast<uintptr_t>(ot)) & 15) == 0;
    long long run = base + (sbeg ? markers_before<B>(tw, twords, cnt, sbeg, lane) : 0u);
    for (int s0 = sbeg; s0 < send; s0 += K4_SEG * k4_unroll<T>()) {
      F field[k4_unroll<T>()];
      T pv[k4_unroll<T>()][4];
#pragma unroll
      for (int u = 0; u < k4_unroll<T>(); ++u) {
        const int sb0 = s0 + u * K4_SEG;
        const int e0 = sb0 + 4 * lane;
        field[u] = sb0 < send ? load_field<B>(tw, twords, (sb0 / K4_SEG) * FB, lane) : (F)0;
        if (vec && sb0 + K4_SEG <= e_hi) {
          ld4(pt + e0, pv[u]);
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            pv[u][k] = (e0 + k >= e_lo && e0 + k < e_hi) ? __ldcs(pt + e0 + k) : (T)0;
        }
      }
#pragma unroll
      for (int u = 0; u < k4_unroll<T>(); ++u) {
        const int sb0 = s0 + u * K4_SEG;
        if (sb0 >= send) break;                  // uniform across the warp
        const int e0 = sb0 + 4 * lane;
        T r[4];
        const unsigned total = decode_step<T, B>(field[u], pv[u], e0, cnt, e_lo, e_hi, run, lt, s_m,
                                                 centres, exact_u, n_inc, A, r);
        run += total;
        if (vec && sb0 + K4_SEG <= e_hi) {
          st4(ot + e0, r);
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (e0 + k >= e_lo && e0 + k < e_hi) ot[e0 + k] = r[k];
        }
      }
    }
    if (send == cnt && lane == 0) {             // this warp ends the tile: all its markers seen
      const long long next = (gt + 1 < g.nsub) ? sub_off[gt + 1] : n_inc;
      if (run != next) report(A, NUMARCK_ERR_CORRUPT);
    }
  }
}

template <typename T, int B = 1>
__device__ __forceinline__ void decode_dispatch(const DecodeArgs& A, const Geometry& g,
                                                long long n_inc, long long g0, long long g1,
                                                const T* s_m) {
  if constexpr (B <= NUMARCK_MAX_B) {
    if (g.B == B)
      decode_tiles<T, B>(A, g, n_inc, g0, g1, s_m);
    else
      decode_dispatch<T, B + 1>(A, g, n_inc, g0, g1, s_m);
  }
}

__global__ void __launch_bounds__(K4_THREADS, 2) k4_decode(DecodeArgs A) {
  __shared__ __align__(16) unsigned char s_tab[DM_SMEM * 8];   // multipliers m = 1 + centre
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
    if (!rc && A.dtype && A.dtype != s_h.dtype) rc = NUMARCK_ERR_INVALID_ARG;
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
    if (rc && blockIdx.x == 0) report(A, rc);
    s_ok = rc == 0 && ((g1 - g0 + 1) << A.seg_log2) > (long long)blockIdx.x * K4_WARPS;
    s_g = g;
    s_g0 = g0;
    s_g1 = g1;
  }
  __syncthreads();
  if (!s_ok) return;
  const Geometry g = s_g;
  const int nm = min(1 << g.B, DM_SMEM);
  if (g.dtype == NUMARCK_F64) {
    double* s_m = reinterpret_cast<double*>(s_tab);
    const double* centres = reinterpret_cast<const double*>(A.blob + g.off_centres);
    for (int r = threadIdx.x; r < nm; r += K4_THREADS) s_m[r] = t_add(1.0, centres[r]);
    __syncthreads();   // the only block-wide barrier after the header
    decode_dispatch<double>(A, g, s_h.n_inc, s_g0, s_g1, s_m);
  } else {
    float* s_m = reinterpret_cast<float*>(s_tab);
    const float* centres = reinterpret_cast<const float*>(A.blob + g.off_centres);
    for (int r = threadIdx.x; r < nm; r += K4_THREADS) s_m[r] = t_add(1.0f, centres[r]);
    __syncthreads();
    decode_dispatch<float>(A, g, s_h.n_inc, s_g0, s_g1, s_m);
  }
}

}  // namespace

cudaError_t launch_decode(const DecodePlan& P, cudaStream_t s) {
  if (P.count <= 0) return cudaSuccess;
  static int occ[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  int per_sm = dev < 64 ? occ[dev] : 0;
  if (per_sm == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k4_decode, K4_THREADS, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (dev < 64) occ[dev] = per_sm;
  }
  long long blocks = (long long)P.sms * per_sm;
  // sub-blocks touched (exact with a host header; else the fewest the range can touch)
  const long long tiles = P.ntiles_hint > 0 ? P.ntiles_hint : (P.count + SUB - 1) / SUB;
  // (with `concurrency` decodes sharing the GPU, each can count on its share of the warps)
  const int sl = seg_log2_for(tiles, blocks * K4_WARPS / std::max(1, P.concurrency));
  if (P.ntiles_hint > 0) {
    const long long need = ((P.ntiles_hint << sl) + K4_WARPS - 1) / K4_WARPS;
    if (blocks > need) blocks = need;
  }
  DecodeArgs A{P.blob, P.prev_seg, P.out_seg, P.status, P.start, P.count, P.n_expected, P.status2,
               P.dtype, sl};
  k4_decode<<<(int)blocks, K4_THREADS, 0, s>>>(A);
  return cudaGetLastError();
}

}  // namespace nmk
