// k4.cuh — the pieces of K4 (decompression, §III.E with Eq. 4 read as R = prev * (1 + centre))
// shared by the decode kernel (k_decode.cu) and the fused decompress-and-classify kernel
// (k_step.cu): vector loads and stores, the B-bit field of a lane in a 128-element step, the
// decode of one step, and the split of a sub-block between warps for small variables.
#pragma once

#include <type_traits>

#include "launch.h"

namespace nmk {

struct DecodeArgs {
  const unsigned char* blob;
  const void* prev_seg;
  void* out_seg;
  int32_t* status;
  long long start, count, n_expected;
  int* status2;              // a second error word (the next compression's), or null
  int dtype;                 // NUMARCK_F32 / NUMARCK_F64 the blob must hold, or 0 for either
  int seg_log2;              // each sub-block is decoded by 2^seg_log2 warps (see seg_log2_for)
};

// An error found on the device goes to both status words (either may be null).
__device__ __forceinline__ void report(const DecodeArgs& A, int rc) {
  if (A.status) atomicExch(A.status, rc);
  if (A.status2) atomicExch(A.status2, rc);
}

template <typename T>
struct BitsOf;
template <>
struct BitsOf<float> {
  using U = unsigned int;
  __device__ __forceinline__ static float as(U u) { return __uint_as_float(u); }
};
template <>
struct BitsOf<double> {
  using U = unsigned long long;
  __device__ __forceinline__ static double as(U u) { return __longlong_as_double((long long)u); }
};

// Four consecutive T as 16-byte vectors (16-byte aligned addresses).
__device__ __forceinline__ void ld4(const double* p, double* v) {
  const double2 a = __ldcs(reinterpret_cast<const double2*>(p));
  const double2 b = __ldcs(reinterpret_cast<const double2*>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void ld4(const float* p, float* v) {
  const float4 a = __ldcs(reinterpret_cast<const float4*>(p));
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void st4(double* p, const double* v) {
  __stcs(reinterpret_cast<double2*>(p), make_double2(v[0], v[1]));
  __stcs(reinterpret_cast<double2*>(p) + 1, make_double2(v[2], v[3]));
}
__device__ __forceinline__ void st4(float* p, const float* v) {
  __stcs(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
}

constexpr int K4_WARPS = 16;                    // warps per CTA (each owns a sub-block or a part)
constexpr int K4_THREADS = K4_WARPS * 32;
constexpr int K4_SEG = 128;                     // elements per warp step: 4 consecutive per lane
// steps whose loads are in flight together: float32 moves half the bytes per load, so it
// keeps two steps in flight to have as many bytes outstanding as float64 with one
template <typename T>
__host__ __device__ constexpr int k4_unroll() { return sizeof(T) == 4 ? 2 : 1; }

template <int B>
struct Field {
  using type = typename std::conditional<(4 * B <= 32), unsigned, unsigned long long>::type;
};

// The 4B-bit field of lane `lane` in the step whose image starts at word ws of the tile image
// tw (twords words). Words past the image read as 0.
template <int B>
__device__ __forceinline__ typename Field<B>::type load_field(const unsigned* tw, int twords,
                                                              int ws, int lane) {
  constexpr int FB = 4 * B;
  using F = typename Field<B>::type;
  if constexpr (FB == 32) {
    const int w = ws + lane;
    return w < twords ? __ldg(tw + w) : 0u;
  } else if constexpr (FB == 64) {
    const int w = ws + 2 * lane;                 // twords is even: both words or neither
    if (w >= twords) return 0ull;
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(tw + w));
    return (unsigned long long)v.x | ((unsigned long long)v.y << 32);
  } else {
    const int bit = FB * lane;
    const int w0 = ws + (bit >> 5), o = bit & 31;
    const unsigned a0 = w0 < twords ? __ldg(tw + w0) : 0u;
    const unsigned a1 = (o + FB > 32 && w0 + 1 < twords) ? __ldg(tw + w0 + 1) : 0u;
    const unsigned long long v = (unsigned long long)a0 | ((unsigned long long)a1 << 32);
    if constexpr (FB > 32) {
      const unsigned a2 = (o + FB > 64 && w0 + 2 < twords) ? __ldg(tw + w0 + 2) : 0u;
      return (F)((v >> o) | (o ? ((unsigned long long)a2 << (64 - o)) : 0ull));
    } else {
      return (F)(v >> o);
    }
  }
}


// Warps per sub-block. A warp decodes its part of a sub-block in 128-point steps, each one a
// dependent round trip to memory (the fields and prev, then the incompressible values), so with
// few sub-blocks (small variables) one warp per sub-block leaves most of the GPU idle and runs a
// 32-step chain. Splitting a sub-block into 2^seg_log2 segments gives each warp 32 >> seg_log2
// steps; a warp that starts inside a sub-block first counts the markers before its segment
// (markers_before: loads that do not depend on each other), which is where its incompressible
// values start. Chosen so that the units (sub-block segments) fill the resident warps.
__host__ __forceinline__ int seg_log2_for(long long tiles, long long resident_warps) {
  int s = 0;
  while (s < 3 && (tiles << s) < resident_warps) ++s;
  return s;
}

// Four consecutive values from shared memory (16-byte aligned).
__device__ __forceinline__ void lds4(const double* p, double* v) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void lds4(const float* p, float* v) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}

// K4's per-warp stage (B <= K4_STAGE_MAX_B): a step's 128 prev values, then its 16 B bytes of
// index field (K4_STAGE_BYTES: room for float64).
constexpr int K4_STAGE_MAX_B = 10;
template <typename T>
__host__ __device__ constexpr int k4_stage_field() { return K4_SEG * (int)sizeof(T); }
constexpr int K4_STAGE_BYTES = K4_SEG * 8 + 16 * K4_STAGE_MAX_B;

// load_field for a staged step: the 4B-bit field of lane `lane` from the step's own 4B words.
template <int B>
__device__ __forceinline__ typename Field<B>::type load_field_staged(const unsigned* sw, int lane) {
  constexpr int FB = 4 * B;
  constexpr int NW = B * 4;                      // words of one step's image
  using F = typename Field<B>::type;
  if constexpr (FB == 32) {
    return sw[lane];
  } else {
    static_assert(FB < 64, "staged steps have B <= 10");
    const int bit = FB * lane;
    const int w0 = bit >> 5, o = bit & 31;
    const unsigned a0 = sw[w0];
    const unsigned a1 = (o + FB > 32 && w0 + 1 < NW) ? sw[w0 + 1] : 0u;
    const unsigned long long v = (unsigned long long)a0 | ((unsigned long long)a1 << 32);
    if constexpr (FB > 32) {
      const unsigned a2 = (o + FB > 64 && w0 + 2 < NW) ? sw[w0 + 2] : 0u;
      return (F)((v >> o) | (o ? ((unsigned long long)a2 << (64 - o)) : 0ull));
    } else {
      return (F)(v >> o);
    }
  }
}

// Number of incompressible points (fields equal to the marker M) among the first e_end points
// of a sub-block (e_end a multiple of K4_SEG, at most its point count cnt); warp-uniform.
template <int B>
__device__ __forceinline__ unsigned markers_before(const unsigned* tw, int twords, int cnt,
                                                   int e_end, int lane) {
  constexpr int FB = 4 * B;
  constexpr unsigned M = (1u << B) - 1u;
  unsigned c = 0;
#pragma unroll 4
  for (int s0 = 0; s0 < e_end; s0 += K4_SEG) {
    const typename Field<B>::type field = load_field<B>(tw, twords, (s0 / K4_SEG) * FB, lane);
    const int e0 = s0 + 4 * lane;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      c += (e0 + k < cnt && ((unsigned)(field >> (k * B)) & M) == M) ? 1u : 0u;
  }
  return __reduce_add_sync(0xffffffffu, c);
}

// One 128-point step of a decode, lane l holding points e0 .. e0+3 (e0 = step start + 4l): their
// indices from the lane's 4B-bit field, the step's incompressible points numbered in element
// order across the warp (four ballots: the lanes before this one, then this lane's earlier
// points) from position `run` of the incompressible table, and r[k] = prev * m[idx] (Eq. 4) or
// the stored value. Points at or past cnt are not counted. An incompressible point whose
// position lies past n_inc reads 0 and, when it lies in [e_lo, e_hi), reports corruption.
// Returns the step's count of incompressible points (the same in every lane).
template <typename T, int B>
__device__ __forceinline__ unsigned decode_step(typename Field<B>::type field, const T (&pv)[4],
                                                int e0, int cnt, int e_lo, int e_hi,
                                                long long run, unsigned lt, const T* s_m,
                                                const T* centres,
                                                const typename BitsOf<T>::U* exact_u,
                                                long long n_inc, const DecodeArgs& A, T (&r)[4]) {
  using U = typename BitsOf<T>::U;
  constexpr unsigned M = (1u << B) - 1u;
  unsigned id[4];
  unsigned nib = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    id[k] = (unsigned)(field >> (k * B)) & M;
    nib |= (e0 + k < cnt && id[k] == M) ? (1u << k) : 0u;
  }
  unsigned before = 0, total = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const unsigned bk = __ballot_sync(0xffffffffu, (nib >> k) & 1u);
    before += __popc(bk & lt);
    total += __popc(bk);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if ((nib >> k) & 1u) {
      const long long pos = run + before + __popc(nib & ((1u << k) - 1u));
      U v = 0;
      if (pos < n_inc) v = exact_u[pos];
      else if (e0 + k >= e_lo && e0 + k < e_hi) report(A, NUMARCK_ERR_CORRUPT);
      r[k] = BitsOf<T>::as(v);
    } else {
      T m;
      if constexpr ((1 << B) <= DM_SMEM) m = s_m[id[k]];
      else m = id[k] < (unsigned)DM_SMEM ? s_m[id[k]] : t_add((T)1, centres[id[k]]);
      r[k] = t_mul(pv[k], m);
    }
  }
  return total;
}

}  // namespace nmk
