// k_zlib.cu — lossless compression of the index table (§IV.C: "NUMARCK splits the index table
// into blocks of same size and compresses each block using the ZLIB"), as zlib streams (RFC
// 1950) of DEFLATE data (RFC 1951) that any inflater reads, and the matching GPU inflater.
//
// Stream layout of index block q (the block's ceil(count * B / 8) bytes, without the 16-byte
// padding of the raw blob):
//   0x78 0x01                                       zlib header (deflate, 32 KB window)
//   for each 4096-element sub-block t of the block:
//     one fixed-Huffman DEFLATE block (BFINAL 0) of t's bytes, then an empty stored block
//     (BFINAL 0, BTYPE 00, LEN 0, NLEN 0xFFFF) that ends t's data on a byte boundary
//   0x03 0x00                                       empty fixed-Huffman block with BFINAL 1
//   Adler-32 of the block's bytes, big-endian
// Matches never reach before the start of their sub-block, so every sub-block's data can be
// inflated on its own from its byte offset: a partial decompression inflates only the
// sub-blocks it decodes (the economics of Table 7).
//
// Match finding: a run of equal B-bit indices repeats the byte pattern with period
// p = B / gcd(B, 8) bytes (1 for B = 8, 5 for B = 10, ...), so LZ77 matches are taken at
// distance p only. A warp encodes one sub-block: lane l parses the l-th 1/32 of its bytes
// greedily (a match of length >= 3 where the bytes equal those p before, else a literal;
// matches stop at the lane's chunk end), the lanes' bit counts are scanned, and each lane writes
// its codes at its bit offset. Z1 counts bits and Adler-32 partial sums, Z2 scans the sizes into
// offsets, Z3 writes the streams; Z4 inflates sub-blocks.
#include <cstring>

#include "launch.h"

namespace nmk {

namespace {

constexpr int ZW = 2;                             // warps per CTA (one sub-block each)
constexpr int ZT = ZW * 32;
constexpr int Z_IN = SUB / 8 * NUMARCK_MAX_B;     // largest sub-block image (bytes)
constexpr int Z_OUT_WORDS = (Z_IN * 9 + 64 + 31) / 32 + 4;   // all literals of 9 bits + tail
constexpr unsigned ADLER = 65521u;
static_assert(sizeof(numarck_zindex_header) == NUMARCK_ZINDEX_HEADER_BYTES, "container header");

// RFC 1951 §3.2.5: length codes 257..285 (base length, extra bits).
__constant__ unsigned short c_len_base[29] = {3,  4,  5,  6,  7,  8,  9,  10, 11,  13,
                                              15, 17, 19, 23, 27, 31, 35, 43, 51,  59,
                                              67, 83, 99, 115, 131, 163, 195, 227, 258};
__constant__ unsigned char c_len_extra[29] = {0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 2, 2, 2,
                                              2, 3, 3, 3, 3, 4, 4, 4, 4, 5, 5, 5, 5, 0};
// distance codes 0..29 (base, extra bits)
__constant__ unsigned short c_dist_base[30] = {1,    2,    3,    4,    5,    7,     9,    13,
                                               17,   25,   33,   49,   65,   97,    129,  193,
                                               257,  385,  513,  769,  1025, 1537,  2049, 3073,
                                               4097, 6145, 8193, 12289, 16385, 24577};
__constant__ unsigned char c_dist_extra[30] = {0, 0, 0, 0, 1, 1, 2, 2, 3,  3,  4,  4,  5,  5,  6,
                                               6, 7, 7, 8, 8, 9, 9, 10, 10, 11, 11, 12, 12, 13, 13};

__device__ __forceinline__ unsigned rev(unsigned code, int len) {
  return __brev(code) >> (32 - len);
}

// Fixed Huffman code of a literal/length symbol (RFC 1951 §3.2.6), bit-reversed for the
// LSB-first stream; *len receives its length.
__device__ __forceinline__ unsigned fixed_code(unsigned sym, int* len) {
  if (sym < 144) { *len = 8; return rev(0x30u + sym, 8); }
  if (sym < 256) { *len = 9; return rev(0x190u + (sym - 144), 9); }
  if (sym < 280) { *len = 7; return rev(sym - 256, 7); }
  *len = 8;
  return rev(0xC0u + (sym - 280), 8);
}

__device__ __forceinline__ int len_code(int len) {   // index into c_len_base
  int c = 0;
  while (c < 28 && c_len_base[c + 1] <= len) ++c;
  return c;
}
__device__ __forceinline__ int dist_code(int d) {
  int c = 0;
  while (c < 29 && c_dist_base[c + 1] <= d) ++c;
  return c;
}

// Bits of a match (length len >= 3, distance d): length code, extra bits, distance code, extra.
__device__ __forceinline__ int match_bits(int len, int d) {
  const int lc = len_code(len), dc = dist_code(d);
  int l;
  fixed_code(257 + lc, &l);
  return l + c_len_extra[lc] + 5 + c_dist_extra[dc];
}

struct BitWriter {
  unsigned* w;        // shared words (zeroed)
  int pos;            // bit position
  __device__ __forceinline__ void put(unsigned v, int n) {   // n <= 25 bits, LSB first
    if (n == 0) return;
    const int wi = pos >> 5, sh = pos & 31;
    atomicOr(&w[wi], v << sh);
    if (sh + n > 32) atomicOr(&w[wi + 1], v >> (32 - sh));
    pos += n;
  }
};

struct ZArgs {
  const unsigned char* blob;
  Geometry g;
  unsigned char* z;          // container
  int64_t* tile_bytes;       // per sub-block: its slot's bytes (Z1), then its offset (Z2)
  unsigned* adler_a;         // per sub-block: sum of bytes mod 65521
  unsigned* adler_w;         // per sub-block: sum of (size - j) * byte_j mod 65521
  numarck_zindex_header zh;  // container header (written into the container by Z2)
};

// The sub-block's image: tile gt of the blob (bytes [0, tb)).
struct ZTile {
  const unsigned char* src;
  int tb;                    // ceil(cnt * B / 8)
  bool first, last;          // first / last sub-block of its index block
  long long q, t;
};
__device__ __forceinline__ ZTile ztile(const ZArgs& A, long long gt) {
  const Geometry& g = A.g;
  ZTile z;
  z.q = gt / g.spb;
  z.t = gt - z.q * g.spb;
  const long long j0 = z.q * g.epb + z.t * SUB;
  const long long bend = min((long long)g.n, (long long)((z.q + 1) * g.epb));
  const int cnt = (int)min((long long)SUB, bend - j0);
  z.tb = (cnt * g.B + 7) / 8;
  z.src = A.blob + g.off_index + z.q * g.block_stride + z.t * (long long)(SUB / 8 * g.B);
  z.first = z.t == 0;
  z.last = j0 + cnt == bend;
  return z;
}

// Greedy parse of bytes [c0, c1) of s with matches at distance p; bits of the codes, and (when
// bw is given) the codes themselves.
__device__ int parse_chunk(const unsigned char* s, int c0, int c1, int p, BitWriter* bw) {
  int bits = 0;
  int i = c0;
  while (i < c1) {
    int len = 0;
    if (i >= p) {
      while (i + len < c1 && len < 258 && s[i + len] == s[i + len - p]) ++len;
    }
    if (len >= 3) {
      const int lc = len_code(len), dc = dist_code(p);
      if (bw) {
        int l;
        const unsigned code = fixed_code(257 + lc, &l);
        bw->put(code, l);
        bw->put((unsigned)(len - c_len_base[lc]), c_len_extra[lc]);
        bw->put(rev((unsigned)dc, 5), 5);
        bw->put((unsigned)(p - c_dist_base[dc]), c_dist_extra[dc]);
      }
      bits += match_bits(len, p);
      i += len;
    } else {
      int l;
      const unsigned code = fixed_code(s[i], &l);
      if (bw) bw->put(code, l);
      bits += l;
      ++i;
    }
  }
  return bits;
}

__device__ __forceinline__ int period_of(int B) {
  int a = B, b = 8;
  while (b) { const int t = a % b; a = b; b = t; }
  return B / a;
}

// Bytes of a sub-block's slot: its DEFLATE data (3 header bits, codes, end-of-block, then the
// empty stored block: 3 bits, padding, 4 bytes), plus the zlib header before the first
// sub-block of a block and the final block and Adler-32 after the last.
__device__ __forceinline__ long long slot_bytes(int code_bits, bool first, bool last) {
  const int bits = 3 + code_bits + 7 + 3;
  return (bits + 7) / 8 + 4 + (first ? 2 : 0) + (last ? 6 : 0);
}

// Z1: per sub-block, the slot size and the Adler-32 partial sums.
__global__ void __launch_bounds__(ZT) z1_size(ZArgs A) {
  __shared__ __align__(16) unsigned char s_in[ZW][Z_IN];
  const int lane = (int)lane_id(), warp = (int)(threadIdx.x >> 5);
  const int p = period_of(A.g.B);
  unsigned char* s = s_in[warp];
  for (long long gt = (long long)blockIdx.x * ZW + warp; gt < A.g.nsub;
       gt += (long long)gridDim.x * ZW) {
    const ZTile z = ztile(A, gt);
    for (int i = lane; i < z.tb; i += 32) s[i] = z.src[i];
    __syncwarp();
    const int per = (z.tb + 31) / 32;
    const int c0 = min(z.tb, lane * per), c1 = min(z.tb, c0 + per);
    int bits = parse_chunk(s, c0, c1, p, nullptr);
    unsigned a = 0;
    unsigned long long w = 0;
    for (int i = lane; i < z.tb; i += 32) {
      a += s[i];
      w += (unsigned long long)(z.tb - i) * s[i];
    }
    bits = __reduce_add_sync(0xffffffffu, bits);
    a = __reduce_add_sync(0xffffffffu, a);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (lane == 0) {
      A.tile_bytes[gt] = slot_bytes(bits, z.first, z.last);
      A.adler_a[gt] = a % ADLER;
      A.adler_w[gt] = (unsigned)(w % ADLER);
    }
    __syncwarp();
  }
}

// Z2: exclusive scan of the slot sizes (one CTA), per-block stream offsets, container header.
__global__ void __launch_bounds__(1024) z2_scan(ZArgs A) {
  __shared__ long long s_w[33];
  __shared__ long long s_carry;
  const Geometry& g = A.g;
  const int tid = (int)threadIdx.x, lane = (int)lane_id(), w = tid >> 5;
  int64_t* zoff = reinterpret_cast<int64_t*>(A.z + A.zh.off_zoff);
  int64_t* sub_zoff = reinterpret_cast<int64_t*>(A.z + A.zh.off_sub_zoff);
  const long long data0 = A.zh.off_data;
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (long long base = 0; base < g.nsub; base += 1024) {
    const long long i = base + tid;
    const long long v = i < g.nsub ? A.tile_bytes[i] : 0;
    long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long u = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += u;
    }
    if (lane == 31) s_w[w] = inc;
    __syncthreads();
    if (w == 0) {
      const long long x = s_w[lane];
      long long xi = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, xi, o);
        if (lane >= o) xi += u;
      }
      s_w[lane] = xi - x;
      if (lane == 31) s_w[32] = xi;
    }
    __syncthreads();
    if (i < g.nsub) {
      const long long off = data0 + s_carry + s_w[w] + inc - v;   // start of this slot
      const long long q = i / g.spb, t = i - q * g.spb;
      A.tile_bytes[i] = off;
      sub_zoff[i] = off + (t == 0 ? 2 : 0);                        // the sub-block's DEFLATE data
      if (t == 0) zoff[q] = off;
    }
    __syncthreads();
    if (tid == 0) s_carry += s_w[32];
    __syncthreads();
  }
  if (tid == 0) {
    zoff[g.nblocks] = data0 + s_carry;
    const numarck_zindex_header h = A.zh;
    const uint4* src = reinterpret_cast<const uint4*>(&h);
    uint4* dst = reinterpret_cast<uint4*>(A.z);
#pragma unroll
    for (int i = 0; i < NUMARCK_ZINDEX_HEADER_BYTES / 16; ++i) dst[i] = src[i];
  }
}

// Z3: writes every slot (zlib header, the sub-block's DEFLATE data, stream trailer).
__global__ void __launch_bounds__(ZT) z3_write(ZArgs A) {
  __shared__ __align__(16) unsigned char s_in[ZW][Z_IN];
  __shared__ __align__(16) unsigned s_out[ZW][Z_OUT_WORDS];
  const int lane = (int)lane_id(), warp = (int)(threadIdx.x >> 5);
  const int p = period_of(A.g.B);
  unsigned char* s = s_in[warp];
  unsigned* o = s_out[warp];
  for (long long gt = (long long)blockIdx.x * ZW + warp; gt < A.g.nsub;
       gt += (long long)gridDim.x * ZW) {
    const ZTile z = ztile(A, gt);
    for (int i = lane; i < z.tb; i += 32) s[i] = z.src[i];
    for (int i = lane; i < Z_OUT_WORDS; i += 32) o[i] = 0u;
    __syncwarp();
    const int per = (z.tb + 31) / 32;
    const int c0 = min(z.tb, lane * per), c1 = min(z.tb, c0 + per);
    const int bits = parse_chunk(s, c0, c1, p, nullptr);
    int incl = bits;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += u;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    BitWriter bw{o, 3 + incl - bits};
    if (lane == 0) {
      BitWriter hw{o, 0};
      hw.put(2u, 3);                       // BFINAL 0, BTYPE 01 (fixed Huffman)
    }
    parse_chunk(s, c0, c1, p, &bw);
    __syncwarp();
    int end_bits = 3 + total;
    if (lane == 0) {
      BitWriter ew{o, end_bits};
      ew.put(0u, 7);                       // end of block (symbol 256)
      ew.put(0u, 3);                       // BFINAL 0, BTYPE 00 (stored), LEN 0 follows
    }
    __syncwarp();
    end_bits += 10;
    const int nb = (end_bits + 7) / 8;     // bytes of codes, padded to a byte boundary
    const long long off = A.tile_bytes[gt];
    unsigned char* dst = A.z + off;
    int k = 0;
    if (z.first) {
      if (lane == 0) { dst[0] = 0x78; dst[1] = 0x01; }
      k = 2;
    }
    const unsigned char* ob = reinterpret_cast<const unsigned char*>(o);
    for (int i = lane; i < nb; i += 32) dst[k + i] = ob[i];
    if (lane == 0) {
      unsigned char* tail = dst + k + nb;
      tail[0] = 0x00; tail[1] = 0x00; tail[2] = 0xFF; tail[3] = 0xFF;   // LEN 0, NLEN 0xFFFF
      if (z.last) {
        tail[4] = 0x03; tail[5] = 0x00;    // empty fixed-Huffman block with BFINAL 1
        // Adler-32 of the block: combine its sub-blocks' partial sums in order
        const long long g0 = z.q * A.g.spb;
        unsigned long long sa = 1, sb = 0;
        long long after = 0;               // bytes of the block after the current sub-block
        for (long long u = gt; u >= g0; --u) {
          const ZTile zu = ztile(A, u);
          sa += A.adler_a[u];
          sb += ((unsigned long long)(after % ADLER) * A.adler_a[u] + A.adler_w[u]) % ADLER;
          after += zu.tb;
        }
        // b = sum over bytes of (N - j) * byte_j + N, with N the block size
        sb = (sb + (unsigned long long)(after % ADLER)) % ADLER;
        sa %= ADLER;
        const unsigned ad = (unsigned)((sb << 16) | sa);
        tail[6] = (unsigned char)(ad >> 24); tail[7] = (unsigned char)(ad >> 16);
        tail[8] = (unsigned char)(ad >> 8);  tail[9] = (unsigned char)ad;
      }
    }
    __syncwarp();
  }
}

// Z4: inflate sub-blocks [g0, g1] back into the raw index section of a blob (the fixed-Huffman
// and stored blocks this encoder writes; anything else is reported as NUMARCK_ERR_CORRUPT).
struct InflateArgs {
  const unsigned char* z;
  unsigned char* blob;
  Geometry g;
  long long g0, g1;
  int32_t* status;
  long long zbytes;
};

struct BitReader {
  const unsigned char* p;
  long long pos, end;       // bit position, end (bits)
  __device__ __forceinline__ unsigned peek(int n) const {   // n <= 24
    const long long byte = pos >> 3;
    unsigned v = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if ((byte + k) * 8 < end) v |= (unsigned)p[byte + k] << (8 * k);
    return (v >> (pos & 7)) & ((1u << n) - 1u);
  }
  __device__ __forceinline__ unsigned get(int n) {
    const unsigned v = n ? peek(n) : 0u;
    pos += n;
    return v;
  }
};

// Decodes one fixed-Huffman literal/length symbol; -1 if invalid.
__device__ __forceinline__ int fixed_symbol(BitReader& br) {
  const unsigned c7 = rev(br.peek(7), 7);
  if (c7 <= 23) { br.pos += 7; return 256 + (int)c7; }
  const unsigned c8 = rev(br.peek(8), 8);
  if (c8 >= 0x30 && c8 <= 0xBF) { br.pos += 8; return (int)(c8 - 0x30); }
  if (c8 >= 0xC0 && c8 <= 0xC7) { br.pos += 8; return 280 + (int)(c8 - 0xC0); }
  const unsigned c9 = rev(br.peek(9), 9);
  if (c9 >= 0x190) { br.pos += 9; return 144 + (int)(c9 - 0x190); }
  return -1;
}

__global__ void __launch_bounds__(128) z4_inflate(InflateArgs A, const int64_t* sub_zoff) {
  const long long gt = A.g0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gt > A.g1) return;
  const Geometry& g = A.g;
  const long long q = gt / g.spb, t = gt - q * g.spb;
  const long long j0 = q * g.epb + t * SUB;
  const long long bend = min((long long)g.n, (long long)((q + 1) * g.epb));
  const int cnt = (int)min((long long)SUB, bend - j0);
  const int tb = (cnt * g.B + 7) / 8;
  const int padded = 16 * ((cnt * g.B + 127) / 128);
  unsigned char* dst = A.blob + g.off_index + q * g.block_stride + t * (long long)(SUB / 8 * g.B);
  const long long zo = sub_zoff[gt];
  const long long zend = gt + 1 < g.nsub ? sub_zoff[gt + 1] : A.zbytes;
  int rc = 0;
  if (zo < 0 || zo > zend || zend > A.zbytes) rc = NUMARCK_ERR_CORRUPT;
  BitReader br{A.z + (rc ? 0 : zo), 0, rc ? 0 : (zend - zo) * 8};
  int n = 0;
  if (!rc && br.get(3) != 2u) rc = NUMARCK_ERR_CORRUPT;   // BFINAL 0, BTYPE 01
  while (!rc) {
    if (br.pos > br.end) { rc = NUMARCK_ERR_CORRUPT; break; }
    const int sym = fixed_symbol(br);
    if (sym < 0 || sym > 285) { rc = NUMARCK_ERR_CORRUPT; break; }
    if (sym < 256) {
      if (n >= tb) { rc = NUMARCK_ERR_CORRUPT; break; }
      dst[n++] = (unsigned char)sym;
    } else if (sym == 256) {
      break;
    } else {
      const int lc = sym - 257;
      const int len = c_len_base[lc] + (int)br.get(c_len_extra[lc]);
      const int dc = (int)rev(br.get(5), 5);
      if (dc > 29) { rc = NUMARCK_ERR_CORRUPT; break; }
      const int d = c_dist_base[dc] + (int)br.get(c_dist_extra[dc]);
      if (d > n || n + len > tb) { rc = NUMARCK_ERR_CORRUPT; break; }
      for (int k = 0; k < len; ++k, ++n) dst[n] = dst[n - d];
    }
  }
  if (!rc && n != tb) rc = NUMARCK_ERR_CORRUPT;
  for (int k = tb; k < padded; ++k) dst[k] = 0;       // the raw blob pads images to 16 bytes
  if (rc && A.status) atomicExch(A.status, rc);
}

}  // namespace

int zindex_layout(const Geometry& g, numarck_zindex_header* zh) {
  std::memset(zh, 0, sizeof(*zh));
  zh->magic = NUMARCK_ZINDEX_MAGIC;
  zh->version = 1;
  zh->B = g.B;
  zh->n = g.n;
  zh->nblocks = g.nblocks;
  zh->nsub = g.nsub;
  zh->off_zoff = NUMARCK_ZINDEX_HEADER_BYTES;
  zh->off_sub_zoff = round_up_i64(zh->off_zoff + (g.nblocks + 1) * 8, 16);
  zh->off_data = round_up_i64(zh->off_sub_zoff + g.nsub * 8, 16);
  return NUMARCK_OK;
}

int64_t zindex_bound(const Geometry& g) {
  numarck_zindex_header zh;
  zindex_layout(g, &zh);
  // every byte a 9-bit literal, plus per sub-block 3 + 7 + 3 bits, padding and 4 bytes, plus
  // per block 2 + 6 bytes
  return zh.off_data + g.index_bytes * 9 / 8 + g.nsub * 10 + g.nblocks * 8 + 64;
}

cudaError_t launch_deflate(const unsigned char* blob, const Geometry& g, unsigned char* z,
                           unsigned char* ws, int sms, cudaStream_t s) {
  if (g.nsub == 0) return cudaSuccess;
  ZArgs A;
  A.blob = blob;
  A.g = g;
  A.z = z;
  zindex_layout(g, &A.zh);
  A.tile_bytes = reinterpret_cast<int64_t*>(ws);
  A.adler_a = reinterpret_cast<unsigned*>(ws + g.nsub * 8);
  A.adler_w = A.adler_a + g.nsub;
  long long blocks = (g.nsub + ZW - 1) / ZW;
  if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
  z1_size<<<(int)blocks, ZT, 0, s>>>(A);
  z2_scan<<<1, 1024, 0, s>>>(A);
  z3_write<<<(int)blocks, ZT, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_inflate(const unsigned char* z, long long zbytes, unsigned char* blob,
                           const Geometry& g, long long g0, long long g1, int32_t* status,
                           cudaStream_t s) {
  if (g1 < g0) return cudaSuccess;
  InflateArgs A{z, blob, g, g0, g1, status, zbytes};
  const long long n = g1 - g0 + 1;
  // the sub-block offsets lie at a fixed place of the container (see zindex_layout)
  numarck_zindex_header lay;
  zindex_layout(g, &lay);
  const int64_t* sub_zoff = reinterpret_cast<const int64_t*>(z + lay.off_sub_zoff);
  z4_inflate<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(A, sub_zoff);
  return cudaGetLastError();
}

}  // namespace nmk
