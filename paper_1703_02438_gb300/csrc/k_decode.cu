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

// Starts the copies of the whole step at s1 (16-byte aligned prev and tile image tw) into the
// warp's stage wst: this lane's four prev values and (lanes 0 .. B-1) the step's 16 B bytes of
// index field.
template <typename T, int B>
__device__ __forceinline__ void k4_stage(unsigned char* wst, const T* pt, int s1, int lane,
                                         const unsigned* tw) {
  constexpr int PER = 16 / (int)sizeof(T);       // values per 16-byte copy
  T* sp = reinterpret_cast<T*>(wst);
  const int e = s1 + 4 * lane;
#pragma unroll
  for (int c = 0; c < 4 / PER; ++c) cp_async16(sp + 4 * lane + c * PER, pt + e + c * PER);
  if (lane < B)
    cp_async16(wst + k4_stage_field<T>() + 16 * lane,
               reinterpret_cast<const unsigned char*>(tw) + (s1 / K4_SEG) * 16 * B + 16 * lane);
  cp_async_commit();
}

// Decodes units u_begin, u_begin + W, ... < u_end (unit u: segment u mod 2^seg_log2 of tile
// u >> seg_log2), one warp. With stages (B <= K4_STAGE_MAX_B: K4_STAGE_BYTES of shared memory
// per warp of the CTA) a warp copies the next step's prev values and index field into its
// stage as soon as it has read the current step's, so that they travel while the current step
// waits for its incompressible values.
template <typename T, int B>
__device__ __forceinline__ void decode_tiles(const DecodeArgs& A, const Geometry& g,
                                             long long n_inc, long long u_begin, long long u_end,
                                             long long W, const T* s_m,
                                             unsigned char* stages = nullptr) {
  using U = typename BitsOf<T>::U;
  using F = typename Field<B>::type;
  constexpr int FB = 4 * B;
  const int lane = (int)lane_id();
  const T* centres = reinterpret_cast<const T*>(A.blob + g.off_centres);
  const int64_t* idx_off = reinterpret_cast<const int64_t*>(A.blob + g.off_idx_off);
  const int64_t* sub_off = reinterpret_cast<const int64_t*>(A.blob + g.off_sub_off);
  const U* exact_u = reinterpret_cast<const U*>(A.blob + g.off_exact);
  const unsigned char* index = A.blob + g.off_index;
  const T* prev = static_cast<const T*>(A.prev_seg);
  T* out = static_cast<T*>(A.out_seg);
  const unsigned lt = lanemask_lt();

  const long long seg_lo = A.start, seg_hi = A.start + A.count;
  const int sl = A.seg_log2;                     // units: 2^sl segments per sub-block
  const int seglen = SUB >> sl;
  for (long long u = u_begin; u < u_end; u += W) {
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
    if constexpr (B <= K4_STAGE_MAX_B) {
      if (stages && vec && (reinterpret_cast<uintptr_t>(tw) & 15) == 0) {
        unsigned char* wst = stages + (threadIdx.x >> 5) * K4_STAGE_BYTES;
        const T* sp = reinterpret_cast<const T*>(wst);
        const unsigned* sw = reinterpret_cast<const unsigned*>(wst + k4_stage_field<T>());
        bool staged = false;                     // this step's inputs are in the stage
        for (int s0 = sbeg; s0 < send; s0 += K4_SEG) {
          const int e0 = s0 + 4 * lane;
          const bool whole = s0 + K4_SEG <= e_hi;
          F field;
          T pv[4];
          if (staged) {
            cp_async_wait_all();
            __syncwarp();                        // the field words other lanes copied
            field = load_field_staged<B>(sw, lane);
            lds4(sp + 4 * lane, pv);
          } else if (whole) {
            field = load_field<B>(tw, twords, (s0 / K4_SEG) * FB, lane);
            ld4(pt + e0, pv);
          } else {
            field = load_field<B>(tw, twords, (s0 / K4_SEG) * FB, lane);
#pragma unroll
            for (int k = 0; k < 4; ++k) pv[k] = e0 + k < e_hi ? __ldcs(pt + e0 + k) : (T)0;
          }
          staged = false;
          const int s1 = s0 + K4_SEG;
          if (s1 < send && s1 + K4_SEG <= e_hi) {
            __syncwarp();                        // every lane has read this step's field
            k4_stage<T, B>(wst, pt, s1, lane, tw);
            staged = true;
          }
          T r[4];
          run += decode_step<T, B>(field, pv, e0, cnt, e_lo, e_hi, run, lt, s_m, centres, exact_u,
                                   n_inc, A, r);
          if (whole) {
            st4(ot + e0, r);
          } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
              if (e0 + k < e_hi) ot[e0 + k] = r[k];
          }
        }
        if (send == cnt && lane == 0) {         // this warp ends the tile: all its markers seen
          const long long next = (gt + 1 < g.nsub) ? sub_off[gt + 1] : n_inc;
          if (run != next) report(A, NUMARCK_ERR_CORRUPT);
        }
        continue;
      }
    }
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
                                                long long n_inc, long long u_begin,
                                                long long u_end, long long W, const T* s_m,
                                                unsigned char* stages = nullptr) {
  if constexpr (B <= NUMARCK_MAX_B) {
    if (g.B == B)
      decode_tiles<T, B>(A, g, n_inc, u_begin, u_end, W, s_m, stages);
    else
      decode_dispatch<T, B + 1>(A, g, n_inc, u_begin, u_end, W, s_m, stages);
  }
}

constexpr int K4_DSMEM = K4_WARPS * K4_STAGE_BYTES;   // K4 kernels: dynamic shared memory

__global__ void __launch_bounds__(K4_THREADS, 2) k4_decode(DecodeArgs A) {
  __shared__ __align__(16) unsigned char s_tab[DM_SMEM * 8];   // multipliers m = 1 + centre
  extern __shared__ __align__(16) unsigned char k4_stages[];   // the warps' stages
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
  const long long u0 = (s_g0 << A.seg_log2) + (long long)blockIdx.x * K4_WARPS + (threadIdx.x >> 5);
  const long long u1 = (s_g1 + 1) << A.seg_log2;
  const long long W = (long long)gridDim.x * K4_WARPS;
  if (g.dtype == NUMARCK_F64) {
    double* s_m = reinterpret_cast<double*>(s_tab);
    const double* centres = reinterpret_cast<const double*>(A.blob + g.off_centres);
    for (int r = threadIdx.x; r < nm; r += K4_THREADS) s_m[r] = t_add(1.0, centres[r]);
    __syncthreads();   // the only block-wide barrier after the header
    decode_dispatch<double>(A, g, s_h.n_inc, u0, u1, W, s_m, k4_stages);
  } else {
    float* s_m = reinterpret_cast<float*>(s_tab);
    const float* centres = reinterpret_cast<const float*>(A.blob + g.off_centres);
    for (int r = threadIdx.x; r < nm; r += K4_THREADS) s_m[r] = t_add(1.0f, centres[r]);
    __syncthreads();
    decode_dispatch<float>(A, g, s_h.n_inc, u0, u1, W, s_m, k4_stages);
  }
}

// ---------------------------------------------------------------------------------------
// Fused batch (K6): the decompression of every blob of a batch in one launch. The prep kernel
// (one CTA) validates each blob's header on the device and writes the tile prefix table; the
// decode kernel's CTA b of G takes tiles [b NT / G, (b + 1) NT / G) of the concatenated list
// and, per blob part, loads the header and the multiplier table into shared memory and runs the
// single-blob loop over its tiles with its warps. A blob whose header is invalid (or whose n
// differs from the item's) contributes no tiles and reports its error in the status word.
// ---------------------------------------------------------------------------------------
constexpr int KP_THREADS = 256;

__global__ void __launch_bounds__(KP_THREADS) k4_fused_prep(FusedDecodeArgs D) {
  __shared__ long long s_sum[KP_THREADS / 32 + 1];
  __shared__ long long s_base;
  if (threadIdx.x == 0) { s_base = 0; D.tpre[0] = 0; *D.ticket = 0ull; }
  __syncthreads();
  for (int c0 = 0; c0 < D.count; c0 += KP_THREADS) {
    const int v = c0 + (int)threadIdx.x;
    long long nsub = 0;
    if (v < D.count) {
      numarck_header h;
      const uint4* src = reinterpret_cast<const uint4*>(D.vars[v].blob);
      uint4* dst = reinterpret_cast<uint4*>(&h);
      for (int i = 0; i < NUMARCK_HEADER_BYTES / 16; ++i) dst[i] = src[i];
      Geometry g{};
      int rc = check_header(h, &g);
      if (!rc && h.n != D.vars[v].n) rc = NUMARCK_ERR_INVALID_ARG;
      if (!rc && ((uintptr_t)D.vars[v].prev | (uintptr_t)D.vars[v].out) %
                     (h.dtype == NUMARCK_F64 ? 8u : 4u))
        rc = NUMARCK_ERR_INVALID_ARG;
      if (rc) {
        if (D.status) atomicExch(D.status, rc);
      } else {
        nsub = g.nsub;
      }
    }
    // inclusive block scan of nsub
    const int lane = (int)lane_id(), w = (int)(threadIdx.x >> 5);
    long long inc = nsub;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) s_sum[w] = inc;
    __syncthreads();
    long long before = s_base;
    for (int i = 0; i < w; ++i) before += s_sum[i];
    if (v < D.count) D.tpre[v + 1] = before + inc;
    __syncthreads();
    if (threadIdx.x == KP_THREADS - 1) s_base = before + inc;
    __syncthreads();
  }
}

// The decode kernel hands out chunks of K4_CHUNK consecutive tiles of the list from a counter
// (tiles differ in cost by dtype, B and marker density, so a static split would leave CTAs
// idle); a CTA keeps the header and multiplier table of the blob it last worked on and reloads
// them only when a chunk starts in another blob.
constexpr int K4_CHUNK = 4 * K4_WARPS;

__global__ void __launch_bounds__(K4_THREADS, 2) k4_fused(FusedDecodeArgs D) {
  __shared__ __align__(16) unsigned char s_tab[DM_SMEM * 8];   // multipliers m = 1 + centre
  extern __shared__ __align__(16) unsigned char k4_stages[];   // the warps' stages
  __shared__ __align__(16) numarck_header s_h;
  __shared__ Geometry s_g;
  __shared__ DecodeArgs s_a;
  __shared__ long long s_chunk;
  __shared__ int s_var;
  const long long NT = D.tpre[D.count];
  if (threadIdx.x == 0) s_var = -1;
  for (;;) {
    __syncthreads();   // the previous chunk is done with the shared state
    if (threadIdx.x == 0) s_chunk = (long long)atomicAdd(D.ticket, 1ull);
    __syncthreads();
    const long long lo = s_chunk * K4_CHUNK;
    if (lo >= NT) break;
    const long long hi = min(NT, lo + K4_CHUNK);
    for (int v = find_var(D.tpre, D.count, lo); v < D.count && D.tpre[v] < hi; ++v) {
      const long long base = D.tpre[v];
      const long long t0 = max(lo, base) - base, t1 = min(hi, D.tpre[v + 1]) - base;
      if (t0 >= t1) continue;
      if (v != s_var) {
        __syncthreads();   // every warp is done with the previous blob's tables
        const FusedDecodeVar& V = D.vars[v];
        if (threadIdx.x < NUMARCK_HEADER_BYTES / 16)
          reinterpret_cast<uint4*>(&s_h)[threadIdx.x] =
              reinterpret_cast<const uint4*>(V.blob)[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 0) {
          check_header(s_h, &s_g);   // valid: the prep kernel gave it tiles
          s_a = DecodeArgs{V.blob, V.prev, V.out, D.status, 0, V.n, V.n, nullptr, 0, D.seg_log2};
          s_var = v;   // read again only after the barriers below
        }
        __syncthreads();
        const int nm = min(1 << s_g.B, DM_SMEM);
        if (s_g.dtype == NUMARCK_F64) {
          double* s_m = reinterpret_cast<double*>(s_tab);
          const double* centres = reinterpret_cast<const double*>(V.blob + s_g.off_centres);
          for (int r = threadIdx.x; r < nm; r += K4_THREADS) s_m[r] = t_add(1.0, centres[r]);
        } else {
          float* s_m = reinterpret_cast<float*>(s_tab);
          const float* centres = reinterpret_cast<const float*>(V.blob + s_g.off_centres);
          for (int r = threadIdx.x; r < nm; r += K4_THREADS) s_m[r] = t_add(1.0f, centres[r]);
        }
        __syncthreads();
      }
      const long long u0 = (t0 << D.seg_log2) + (threadIdx.x >> 5), u1 = t1 << D.seg_log2;
      if (s_g.dtype == NUMARCK_F64)
        decode_dispatch<double>(s_a, s_g, s_h.n_inc, u0, u1, K4_WARPS,
                                reinterpret_cast<const double*>(s_tab), k4_stages);
      else
        decode_dispatch<float>(s_a, s_g, s_h.n_inc, u0, u1, K4_WARPS,
                               reinterpret_cast<const float*>(s_tab), k4_stages);
    }
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
    cudaError_t e = cudaFuncSetAttribute(k4_decode, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         K4_DSMEM);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k4_decode, K4_THREADS, K4_DSMEM);
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
  k4_decode<<<(int)blocks, K4_THREADS, K4_DSMEM, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_fused_decode(const FusedDecodeArgs& D, int sms, cudaStream_t s) {
  if (D.count <= 0) return cudaSuccess;
  static int occ[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  int per_sm = dev < 64 ? occ[dev] : 0;
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k4_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         K4_DSMEM);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k4_fused, K4_THREADS, K4_DSMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (dev < 64) occ[dev] = per_sm;
  }
  k4_fused_prep<<<1, KP_THREADS, 0, s>>>(D);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k4_fused<<<sms * per_sm, K4_THREADS, K4_DSMEM, s>>>(D);
  return cudaGetLastError();
}

}  // namespace nmk
