/*
 * numarck.h — C ABI of the GB300 NUMARCK compression hot path.
 *
 * NUMARCK (Yuan et al., "Parallel Implementation of Lossy Data Compression for Temporal
 * Data Sets", arXiv 1703.02438) compresses a timestep of a variable against the previous
 * timestep of the same variable:
 *
 *   1. change ratios      d_j = (cur_j - prev_j) / prev_j                 (Eq. 1, §III.A)
 *   2. top-k binning      bins of width 2E over the ratios, histogram, keep the
 *                         k = 2^B - 1 most populated bins                  (§IV.B.1)
 *   3. indexing           each point gets the B-bit id of its selected bin, or the
 *                         marker 2^B - 1 ("incompressible"), whose value is stored as is
 *                                                                          (§III.C, §IV.C)
 *   4. decompression      R_j = prev_j * (1 + centre[idx_j]), or the stored value
 *                                                                          (Eq. 4, §III.E)
 *   5. partial decompression of a segment via per-block offset tables       (§IV.C, §V.C)
 *
 * Conventions for every entry point:
 *   - All data pointers (prev, cur, blob, workspace, out) are DEVICE pointers owned by the
 *     caller. The library never allocates device memory and never frees caller memory.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy default stream).
 *     No entry point synchronises the stream except where stated ("synchronous").
 *   - Argument errors are detected on the host before any launch, and the call then
 *     returns without touching device memory. Errors found on the device during
 *     compression are written to the blob header's `status` word (read it with
 *     numarck_blob_size after the stream has been synchronised).
 *   - The element type T is float (dtype NUMARCK_F32) or double (NUMARCK_F64); L = sizeof(T).
 *     All method arithmetic is done in T with IEEE round-to-nearest-even and no fused
 *     multiply-add, in the order stated in the blob format description below, so that the
 *     output is a deterministic function of the inputs (independent of launch shape).
 *   - Multi-byte fields are little-endian.
 */
#ifndef NUMARCK_H
#define NUMARCK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque CUDA stream handle; identical to cudaStream_t / CUstream. */
typedef struct CUstream_st* numarck_stream_t;

/* ---- status codes (return value of every int-returning entry point) ---- */
#define NUMARCK_OK               0
#define NUMARCK_ERR_INVALID_ARG  1  /* bad pointer, size, E, B, dtype, anchor or block size */
#define NUMARCK_ERR_CAPACITY     2  /* blob or workspace buffer smaller than required       */
#define NUMARCK_ERR_CUDA         3  /* a CUDA runtime call or kernel launch failed           */
#define NUMARCK_ERR_CORRUPT      4  /* blob header inconsistent (magic, version, fields)     */
#define NUMARCK_ERR_RANGE        5  /* decompress range outside [0, n]                       */
#define NUMARCK_ERR_TIMEOUT      6  /* a bounded device-side wait gave up                    */
#define NUMARCK_ERR_NOMEM        7  /* host-side allocation failed                           */

/* ---- element types and grid anchors ---- */
#define NUMARCK_F32 0
#define NUMARCK_F64 1

/* Grid origin of the top-k bins (the paper says the ratio range is divided into bins of
 * width 2E, §IV.B.1, and that the global min/max ratio is "used in the bin construction
 * phase", §IV.A, but never states where the first edge lies):
 *   NUMARCK_ANCHOR_ZERO  edges at a + b*2E with a = -E: bin 0 is centred on ratio 0, so
 *                        unchanged points reconstruct exactly (default; no extra pass).
 *   NUMARCK_ANCHOR_MIN   a = the minimum binnable ratio (the paper's literal reading;
 *                        costs one extra pass over both timesteps). */
#define NUMARCK_ANCHOR_ZERO 0
#define NUMARCK_ANCHOR_MIN  1

/* ---- format constants ---- */
#define NUMARCK_MAGIC          0x314B4D4Eu   /* "NMK1" */
#define NUMARCK_VERSION        1u
#define NUMARCK_HEADER_BYTES   256           /* fixed header at the start of every blob   */
#define NUMARCK_SECTION_ALIGN  256           /* every section starts at a multiple of it  */
#define NUMARCK_SUB_BLOCK      4096          /* elements per sub-block (see sub_off below) */
#define NUMARCK_WINDOW_LOG2    21            /* binnable iff |ratio| <= 2^21 * 2E          */
#define NUMARCK_MAX_B          16
#define NUMARCK_DEFAULT_BLOCK_BYTES (1 << 20) /* 1 MB index blocks, as in the paper's runs */

/* Compression parameters (user-controllable parameters of §IV.B.2 and §IV.C). */
typedef struct numarck_params {
  int32_t dtype;        /* NUMARCK_F32 or NUMARCK_F64                                     */
  int32_t B;            /* index bits, 1..16 (k = 2^B - 1 bins, marker M = 2^B - 1), or 0:  *
                         * chosen from the histogram by Eqs. 5-6 (§IV.B.2; see below)     */
  double  E;            /* error bound, 2^-60 <= E < 1; bin width is 2E (§IV.B.1)          */
  int32_t anchor;       /* NUMARCK_ANCHOR_ZERO or NUMARCK_ANCHOR_MIN                      */
  int32_t reserved;     /* must be 0                                                       */
  int64_t block_bytes;  /* index-table block size in bytes, 2..2^30; 0 = the 1 MB default  */
} numarck_params;

/*
 * ---- Blob format (version 1) ----
 *
 * A compressed timestep is one contiguous byte buffer ("blob") holding the arrays of the
 * paper's file layout (§IV.D, Fig. 2): bin centres, the index-table offset table, the
 * incompressible offset table, the big index table and the incompressible table. It adds a
 * fixed header and a sub-block offset table. Sections start at multiples of 256 bytes; all
 * bytes between sections and all padding are zero, so a blob is a pure function of
 * (prev, cur, params).
 *
 *   [0, 256)          header (numarck_header below)
 *   off_centres       T centres[2^B]        centre of the bin with index r (r < n_sel);
 *                                           0 for r >= n_sel (Fig. 2 "bin_centers", 2^B
 *                                           entries, §III.B)
 *   off_idx_off       int64 idx_off[nblocks+1]  byte offset of index block q inside the
 *                                           index section; idx_off[nblocks] = its size (§IV.C)
 *   off_inc_off       int64 inc_off[nblocks+1]  incompressible points in blocks < q;
 *                                           inc_off[nblocks] = n_inc (§IV.C)
 *   off_sub_off       int64 sub_off[nsub]   incompressible points before sub-block g
 *                                           (global count; sub-blocks below)
 *   off_index         index blocks          block q holds the indices of elements
 *                                           [q*epb, min(n, (q+1)*epb)), epb =
 *                                           floor(8*block_bytes / B) (§IV.C); index i of the
 *                                           block occupies bits [i*B, i*B+B) of the block,
 *                                           least significant index bit first, and bit t of
 *                                           the block is bit (t mod 8) of byte t/8. A block
 *                                           is ceil(count*B/8) bytes followed by zero bytes
 *                                           up to a multiple of 16; block q starts at
 *                                           q * block_stride, block_stride =
 *                                           round_up(ceil(epb*B/8), 16).
 *   off_exact         T exact[n_inc]        the values cur_j of the points with index M, in
 *                                           ascending j, bit-for-bit (§III.C)
 *   total_bytes       = off_exact + n_inc * L
 *
 * Sub-blocks: block q is split into ceil(count_q / 4096) sub-blocks of 4096 elements (the
 * last one of a block may be shorter); they are numbered globally in element order,
 * nsub in total. sub_off lets a decoder start at any sub-block without scanning the block
 * (the paper stores only the per-block table, §IV.C; the extra table costs 8 bytes per
 * 4096 elements).
 *
 * Method arithmetic (all in T, RNE, no FMA), with E_T = (T)E:
 *   w = E_T + E_T;  inv_w = 1 / w;  cap = w * 2^21
 *   ratio_j = (cur_j - prev_j) / prev_j                                   (Eq. 1)
 *   binnable_j = ratio_j finite and |ratio_j| <= cap
 *   a = -E_T (ANCHOR_ZERO) | min over binnable ratios, 0 if none (ANCHOR_MIN)
 *   bin_j = floor((ratio_j - a) * inv_w)                                  (§IV.B.1)
 *   histogram over the bins of binnable points; S = the min(k, #non-empty) bins with the
 *   largest counts, ties broken by the smaller bin; index r of a selected bin = its position
 *   in S sorted by ascending bin                                          (§IV.B.1)
 *   centre_r = a + (((T)bin_r + 0.5) * w);  m_r = 1 + centre_r
 *   idx_j = r if binnable, bin_j in S and |(prev_j * m_r) - cur_j| <= E_T * |cur_j|,
 *           else M                                                        (§III.C)
 *   decompression: R_j = idx_j == M ? exact[next] : prev_j * (1 + centre[idx_j])  (Eq. 4)
 */
typedef struct numarck_header {
  uint32_t magic;        /*   0: NUMARCK_MAGIC                                   */
  uint32_t version;      /*   4: NUMARCK_VERSION                                 */
  int32_t  dtype;        /*   8                                                  */
  int32_t  B;            /*  12                                                  */
  double   E;            /*  16: E as passed in numarck_params                   */
  int32_t  anchor;       /*  24                                                  */
  int32_t  status;       /*  28: 0, or a NUMARCK_ERR_* code set on the device    */
  int64_t  n;            /*  32: elements                                        */
  int64_t  block_bytes;  /*  40                                                  */
  int64_t  epb;          /*  48: elements per index block (Fig. 2 "elements_per_block") */
  int64_t  nblocks;      /*  56                                                  */
  int64_t  sub;          /*  64: NUMARCK_SUB_BLOCK                               */
  int64_t  nsub;         /*  72                                                  */
  int64_t  n_sel;        /*  80: selected bins |S| <= 2^B - 1                    */
  int64_t  n_inc;        /*  88: incompressible points                           */
  double   a;            /*  96: grid anchor (the T value, widened exactly)      */
  int64_t  block_stride; /* 104                                                  */
  int64_t  off_centres;  /* 112                                                  */
  int64_t  off_idx_off;  /* 120                                                  */
  int64_t  off_inc_off;  /* 128                                                  */
  int64_t  off_sub_off;  /* 136                                                  */
  int64_t  off_index;    /* 144                                                  */
  int64_t  off_exact;    /* 152                                                  */
  int64_t  total_bytes;  /* 160                                                  */
  uint8_t  reserved[88]; /* 168: zero                                            */
} numarck_header;

/* ---- sizing (host only; never touch the device) ---- */

/* Bytes a blob can need for n elements: every section sized for the worst case n_inc = n
 * (for B = 0: the largest over B = 1..16, i.e. B = 16). Returns 0 if n or *p is invalid. */
size_t numarck_compress_bound(int64_t n, const numarck_params* p);

/* Bytes of device workspace numarck_compress needs for n elements (histogram window of
 * 2^22 + 16 bins, rank table, per-sub-block scan state; for B = 0 sized for B = 16).
 * Returns 0 if invalid. */
size_t numarck_workspace_bytes(int64_t n, const numarck_params* p);

/* Zero-fills a workspace (asynchronous on stream). A workspace must be zero-filled once
 * before its first use; every later numarck_compress call leaves it ready for the next
 * one, so it is initialised once and reused. That holds for a call whose kernels report an
 * error in the blob's status word too; only a call that returns NUMARCK_ERR_CUDA (a kernel
 * that could not be queued) may leave it partly filled, and it is then zero-filled again. Returns NUMARCK_ERR_INVALID_ARG for a NULL
 * pointer, NUMARCK_ERR_CUDA if the memset cannot be queued. */
int numarck_workspace_init(void* ws, size_t ws_bytes, numarck_stream_t stream);

/* ---- compression (§III.A-C, §IV.A-C) ----
 *
 * prev, cur : device arrays of n elements of T (any alignment; 16-byte aligned is faster).
 *             prev is the timestep the decompressor will hold: in a chain of timesteps pass
 *             the previous reconstruction so that errors do not accumulate (Eq. 4 uses
 *             R_{i-1}).
 * n         : 0 <= n <= 2^40.
 * p         : parameters (host pointer).
 * blob      : device buffer of blob_cap >= numarck_compress_bound(n, p) bytes, 256-byte
 *             aligned. On completion it holds the blob; bytes past total_bytes are undefined.
 * ws        : device workspace of ws_bytes >= numarck_workspace_bytes(n, p), 256-byte
 *             aligned, zero-filled before first use (numarck_workspace_init). Two calls
 *             that overlap in time must not share a workspace.
 * stream    : the stream the work is queued on.
 * Returns NUMARCK_OK once the work is queued (host-side errors as listed above).
 *
 * Automatic index length (p->B = 0, §IV.B.2): after the histogram pass the library evaluates
 * file_size(B) = 2^B * L + n * B / 8 + n * alpha(B) * L (Eqs. 5, 6) for B = 1..16, where
 * alpha(B) counts as compressible every point of the 2^B - 1 most populated bins, and keeps
 * the smallest (ties: smaller B). The rest of the layout depends on B, so the call reads the
 * choice back (it synchronises `stream` once) and then queues the remaining kernels; the
 * chosen B is in the blob header. It returns NUMARCK_ERR_INVALID_ARG while `stream` is being
 * captured into a graph, and the batch entry points reject B = 0. */
int numarck_compress(const void* prev, const void* cur, int64_t n, const numarck_params* p,
                     void* blob, size_t blob_cap, void* ws, size_t ws_bytes,
                     numarck_stream_t stream);

/* ---- compression without a workspace argument ----
 * The paper has no counterpart to this entry point; it exists for callers that cannot allocate
 * device memory: a simulation that has handed all of HBM to its own pool (in-situ checkpoint
 * compression), code that must not take the implicit device synchronisation of
 * cudaMalloc/cudaFree, or plugins whose host application forbids raw CUDA allocations.
 *
 * Same arguments, results and errors as numarck_compress, minus the workspace: the scratch
 * memory is one fixed array of NUMARCK_NOALLOC_SCRATCH_BYTES (48 MiB) inside the library's
 * device image. Once the library's device code is loaded on a GPU (at the latest at the first
 * call of this entry point there), that GPU holds the array until the process exits. The call
 * allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 *
 * Limit: (n, p) is accepted only if numarck_workspace_bytes(n, p) <=
 * NUMARCK_NOALLOC_SCRATCH_BYTES; otherwise NUMARCK_ERR_CAPACITY is returned before any launch.
 * The fixed part of the workspace is about 41 MiB; the rest holds 8 bytes per 4096-element
 * sub-block, so with the default 1 MB index blocks n up to about 3.7 * 10^9 elements is
 * accepted; smaller blocks lower the limit.
 *
 * First call on a device: it looks up the array's device address with that device current and
 * clears the whole array on `stream`. Make that first call before any stream capture.
 * Every call shares the one array, which keeps the last call's contents; each call clears the
 * part that must start at zero. Calls that overlap on the GPU (different streams, or several
 * host threads without ordering) race on the array: serialise them. */
#define NUMARCK_NOALLOC_SCRATCH_BYTES (48 * 1024 * 1024)
int numarck_compress_noalloc(const void* prev, const void* cur, int64_t n,
                             const numarck_params* p, void* blob, size_t blob_cap,
                             numarck_stream_t stream);

/* ---- header inspection (host only) ----
 * header_host: a HOST copy of (at least) the first NUMARCK_HEADER_BYTES bytes of a blob,
 * taken after the compressing stream has been synchronised.
 * numarck_blob_size: on success stores total_bytes; returns the device status word if it is
 *   non-zero, NUMARCK_ERR_CORRUPT if magic/version/fields are inconsistent.
 * numarck_read_header: validates and copies the header into *out. */
int numarck_blob_size(const void* header_host, size_t* bytes);
int numarck_read_header(const void* header_host, numarck_header* out);

/* ---- decompression (Eq. 4, §III.E) ----
 * blob        : device pointer to a complete blob (256-byte aligned). The kernel reads the
 *               header from device memory and checks it (magic, version, status word,
 *               geometry); a blob produced by numarck_compress on the same stream may be
 *               decompressed right away, without synchronising.
 * header_host : optional host copy of its header (NUMARCK_HEADER_BYTES). When given, the
 *               header and the arguments are validated on the host before any launch and the
 *               call returns the error code; when NULL, errors found on the device are reported
 *               only through status_dev.
 * prev        : device array of n elements of T, the same prev the blob was compressed
 *               against.
 * out         : device array of n elements of T; receives the reconstruction. Must not
 *               overlap prev or blob.
 * n           : must equal the header's n.
 * status_dev  : optional device int32; if non-NULL the kernel stores a NUMARCK_ERR_* code
 *               into it when the device header is invalid or its status word is set, when n
 *               or the range does not match the header, or when the offset tables disagree
 *               with the index table; nothing is written to out then. It is not cleared on
 *               success. May be NULL.
 */
int numarck_decompress(const void* blob, const void* header_host, const void* prev,
                       void* out, int64_t n, int32_t* status_dev, numarck_stream_t stream);

/* ---- partial decompression (§IV.C, §V.C) ----
 * Reconstructs elements [start, start+count) only, touching the index blocks and exact
 * values of that segment.
 * prev_seg : device array of count elements = prev[start : start+count].
 * out_seg  : device array of count elements; receives R[start : start+count].
 * Returns NUMARCK_ERR_RANGE unless 0 <= start <= start+count <= n (checked on the host when
 * header_host is given, else on the device through status_dev).
 * The result equals the same slice of numarck_decompress's output, bit for bit. */
int numarck_decompress_range(const void* blob, const void* header_host,
                             const void* prev_seg, int64_t start, int64_t count,
                             void* out_seg, int32_t* status_dev, numarck_stream_t stream);

/* ---- one step of a chain of timesteps (Eq. 4, §III.E; Eq. 1, §IV.B, §III.C) ----
 * In a chain every timestep is compressed against the reconstruction of the previous one, so a
 * decompression is followed by a compression whose prev is its output. This call queues both:
 *   numarck_decompress(blob, header_host, prev, out, n, status_dev, stream), then
 *   numarck_compress(out, next_cur, n, p, next_blob, next_blob_cap, ws, ws_bytes, stream),
 * with the same results byte for byte. With the zero-centred grid (p->anchor ==
 * NUMARCK_ANCHOR_ZERO) the decompression and the first pass of the compression (change ratio,
 * bin, own-bin check, histogram) run as one kernel that classifies each reconstructed point
 * while it is in registers, so out is written once and not read back. With
 * NUMARCK_ANCHOR_MIN the grid origin needs the minimum ratio over all of out first, and the two
 * run one after the other.
 * blob, header_host, prev, status_dev : as for numarck_decompress; the blob must hold elements
 *               of p->dtype (checked on the host when header_host is given, else on the
 *               device).
 * out         : device array of n elements of T: receives the reconstruction, which is also
 *               the compression's prev. Must not overlap prev, blob, next_cur, next_blob or ws.
 * next_cur, p, next_blob, next_blob_cap, ws, ws_bytes : as cur, p, blob, blob_cap, ws,
 *               ws_bytes of numarck_compress (next_blob must not be blob).
 * An error that the decompression finds on the device is stored into status_dev (if given)
 * and also into next_blob's header status word, so that the next blob is refused too.
 * Returns NUMARCK_OK once the work is queued, or the host-side errors of either call. */
int numarck_decompress_compress(const void* blob, const void* header_host, const void* prev,
                                void* out, int64_t n, int32_t* status_dev, const void* next_cur,
                                const numarck_params* p, void* next_blob, size_t next_blob_cap,
                                void* ws, size_t ws_bytes, numarck_stream_t stream);

/* ---- batches of variables ----
 * The paper stores several compressed variables in one file (§IV.D); a checkpoint holds many
 * variables of different sizes, types, error bounds and index widths. A batch call compresses
 * (or decompresses) all of them with the kernels of `lanes` variables in flight at once:
 * variables are assigned to lanes longest-first, each lane is a stream of the library forked from
 * `stream` with an event and joined back into it before the call's work completes, and kernel
 * grids are sized for 1/grid_share of the GPU. The results are those of the single-variable
 * entry points, byte for byte. The fork/join consists of event records and waits only, so a batch
 * can be captured into a CUDA graph (make one uncaptured call per device first: it creates the
 * library's lane streams and configures its kernels). Calls of different host threads are
 * serialised inside the library while they are queued. */
typedef struct numarck_batch_item {
  const void* prev;        /* device array of n elements of params.dtype                    */
  const void* cur;         /* device array of n elements of params.dtype                    */
  int64_t n;
  numarck_params params;   /* per-variable dtype, B, E, anchor and block size               */
  void* blob;              /* device buffer, 256-byte aligned                               */
  size_t blob_cap;         /* >= numarck_compress_bound(n, &params)                         */
} numarck_batch_item;

typedef struct numarck_batch_decode_item {
  const void* blob;        /* device pointer to a complete blob (256-byte aligned)          */
  const void* prev;        /* device array of n elements (the prev of the compression)     */
  void* out;               /* device array of n elements; receives the reconstruction      */
  int64_t n;               /* must equal the blob's n                                       */
} numarck_batch_decode_item;

/* Workspace bytes for numarck_compress_batch with this item list and lane count (one slice per
 * lane, each the largest single-variable workspace of its lane). 0 if an item is invalid. */
size_t numarck_batch_workspace_bytes(const numarck_batch_item* items, int count, int lanes);

/* Compresses count variables. ws: device workspace of >= numarck_batch_workspace_bytes bytes,
 * zero-filled before first use (numarck_workspace_init) and reusable with the same item list
 * and lane count (each lane's slice sits at an offset that depends on both: after a change,
 * zero-fill it again). lanes >= 1 (clamped to
 * count and 64), grid_share >= 1. Every item is validated on the host before any launch; the
 * return value is the first item error found (nothing is queued then), else NUMARCK_OK. */
int numarck_compress_batch(const numarck_batch_item* items, int count, int lanes, int grid_share,
                           void* ws, size_t ws_bytes, numarck_stream_t stream);

/* Decompresses count blobs (Eq. 4) with `lanes` in flight; status_dev as in
 * numarck_decompress (shared by all items; may be NULL). */
int numarck_decompress_batch(const numarck_batch_decode_item* items, int count, int lanes,
                             int grid_share, int32_t* status_dev, numarck_stream_t stream);

/* ---- fused batches (one persistent launch per phase over all variables) ----
 * The same results as numarck_compress_batch / numarck_decompress_batch (byte for byte the
 * single-variable results), computed differently: instead of each variable's kernels, every
 * phase of the method runs as ONE launch over a work list held in device memory that
 * concatenates all variables' items (their bytes for the ratio/histogram pass of §III.A and
 * §IV.B.1, one CTA per variable for the top-k selection, their 4096-element tiles for indexing
 * and packing (§III.C, §IV.C) and for the incompressible copy, their scan blocks for the offset
 * tables). Each item's dtype, E, B, anchor and block size come from its variable's descriptor.
 * Every launch fills the GPU regardless of how the batch's sizes are distributed, and a batch
 * is seven launches per group (plus small upload launches) whatever its count.
 *
 * Tuning (NULL: the defaults): k1_threads 512 or 1024 (threads per CTA of the ratio/histogram
 * pass; 0 = 1024), exact_warps 4 or 8 (warps per CTA of the incompressible copy; 0 = 8),
 * decode_seg_log2 0..3 (each 4096-element tile is decoded by 2^decode_seg_log2 warps), groups
 * 1..64 and streams 1..8 (0 = 1 each): the variables are split into `groups` work lists of
 * about equal bytes, each compressed by its own sequence of fused launches, and the groups run
 * on `streams` streams of the library (forked from and joined back into the caller's stream)
 * with every launch sized for 1/streams of the GPU, so that the ALU-bound ratio pass of one group
 * overlaps the memory-bound passes of another. reserved must be 0. The result does not depend
 * on the tuning. */
typedef struct numarck_fused_tuning {
  int32_t k1_threads;
  int32_t exact_warps;
  int32_t decode_seg_log2;
  int32_t groups;
  int32_t streams;
  int32_t reserved;
} numarck_fused_tuning;

/* Workspace bytes of numarck_compress_batch_fused for this item list: 256 bytes of control,
 * the variables' descriptors and work-list tables, and one numarck_workspace_bytes slice per
 * variable (about 41 MiB each). 0 if an item is invalid (B = 0 is rejected: the automatic
 * index length synchronises). */
size_t numarck_fused_workspace_bytes(const numarck_batch_item* items, int count);

/* Compresses count variables with the fused launches. ws: device workspace of
 * >= numarck_fused_workspace_bytes bytes, 256-byte aligned, zero-filled before first use
 * (numarck_workspace_init). A call leaves it ready for the next call with the same item list
 * (the same n and params per position); a workspace that served a different list must be
 * zero-filled again, because each variable's slice sits at an offset that depends on the
 * sizes before it. Every item is validated on the host before any launch; the return value is
 * the first error found (nothing is queued then), else NUMARCK_OK once the work is queued on
 * `stream`. Device-side errors go to each blob's status word as for numarck_compress. The call
 * is a fixed sequence of launches on `stream` (no host synchronisation), so it can be captured
 * into a CUDA graph and replayed with new data in the same buffers. */
int numarck_compress_batch_fused(const numarck_batch_item* items, int count,
                                 const numarck_fused_tuning* tuning, void* ws, size_t ws_bytes,
                                 numarck_stream_t stream);

/* Workspace bytes of numarck_decompress_batch_fused: the blobs' descriptors and tile table. */
size_t numarck_fused_decode_workspace_bytes(int count);

/* Decompresses count blobs (Eq. 4) with one prep launch (the blob headers validated on the
 * device, the tile table built) and one decode launch over all blobs' tiles. ws: device buffer
 * of >= numarck_fused_decode_workspace_bytes(count) bytes, 256-byte aligned (no
 * initialisation needed). status_dev as in numarck_decompress (shared by all items; may be
 * NULL): a blob whose header is invalid or whose n differs from the item's is not decoded and
 * reports its error there. Capturable into a CUDA graph like the compression. */
int numarck_decompress_batch_fused(const numarck_batch_decode_item* items, int count,
                                   const numarck_fused_tuning* tuning, void* ws, size_t ws_bytes,
                                   int32_t* status_dev, numarck_stream_t stream);

/* ---- tracing (kernel-level timing for profilers and benchmarks) ----
 * events : an array of `count` cudaEvent_t handles owned by the caller, or NULL to stop.
 * While set, every numarck_compress call made on this host thread records, on its stream,
 * events[0] before its first kernel and events[1..5] after, in order, the ratio + histogram
 * kernel(s), the top-k kernel, the assign + pack kernel, the offset-table scan and the
 * incompressible-value copy; every numarck_decompress[_range] call records events[0] before and
 * events[1] after its kernel. A call needs count >= 6 (compress) or >= 2 (decompress) to record
 * anything. A numarck_compress_batch_fused call records events[0] before its first launch and
 * events[1..5] after its ratio/histogram, top-k, indexing, offset-scan and incompressible-copy
 * launches; a numarck_decompress_batch_fused call events[0] and events[1] around its launches.
 * Returns NUMARCK_ERR_INVALID_ARG if count < 0. */
int numarck_trace_events(void* const* events, int count);

/* ---- self-test of the bounded device waits ----
 * The only kernel that waits on other CTAs, the incompressible-offset scan (its decoupled
 * look-back, §IV.C offsets), bounds every wait: after 2 s on the GPU's global timer it stores
 * NUMARCK_ERR_TIMEOUT in the blob's status word and finishes, so a flag that is never set cannot
 * hang the GPU. This entry point runs that same wait on a caller's flag: one single-thread
 * kernel waits until the 8-byte word at flag_dev (device, 8-byte aligned) is non-zero, for at
 * most limit_ns nanoseconds once its first 64 polls have failed, then stores NUMARCK_OK or
 * NUMARCK_ERR_TIMEOUT into *status_dev (device int32). The kernel only reads the flag.
 * limit_ns must lie in [1e6, 1e10] (1 ms to 10 s). Returns NUMARCK_ERR_INVALID_ARG for null or
 * misaligned pointers or a limit out of range, NUMARCK_OK once the kernel is queued. */
int numarck_selftest_wait(const void* flag_dev, int64_t limit_ns, int32_t* status_dev,
                          numarck_stream_t stream);

/* Human-readable name of a status code (static string). */
const char* numarck_status_string(int code);

/* Library version string, e.g. "numarck-gb300 1 sm_103a". */
const char* numarck_version(void);

/* ---- lossless index compression (§IV.C: each index block compressed with ZLIB) ----
 *
 * numarck_deflate_index turns a blob's index section into a container of zlib streams (RFC
 * 1950; DEFLATE data of RFC 1951 that any inflater, e.g. zlib's, reads): one stream per index
 * block holding the block's ceil(count * B / 8) bytes (without the raw blob's 16-byte padding).
 * Inside a stream each 4096-element sub-block is one DEFLATE block whose matches stay inside the
 * sub-block: dynamic Huffman (the code built from its index block's symbol counts, repeated in
 * every sub-block's header), fixed Huffman or stored, whichever is smallest; a Huffman block is followed by an empty stored block
 * that ends it on a byte boundary, so any sub-block inflates on its own: numarck_inflate_index restores only the sub-blocks that
 * cover [start, start + count) into a blob buffer (the raw index section, padding included),
 * which numarck_decompress_range then decodes.
 *
 * Container (little-endian): numarck_zindex_header (64 bytes) · int64 zoff[nblocks + 1] at
 * off_zoff (byte offset of index block q's zlib stream; the last entry = total_bytes) · int64
 * sub_zoff[nsub] at off_sub_zoff (byte offset of sub-block t's DEFLATE data) · the streams from
 * off_data on. */
#define NUMARCK_ZINDEX_MAGIC        0x5849414Eu   /* "NAIX" */
#define NUMARCK_ZINDEX_HEADER_BYTES 64

typedef struct numarck_zindex_header {
  uint32_t magic;        /*   0 */
  int32_t  version;      /*   4: 1 */
  int32_t  B;            /*   8 */
  int32_t  pad;          /*  12 */
  int64_t  n;            /*  16 */
  int64_t  nblocks;      /*  24 */
  int64_t  nsub;         /*  32 */
  int64_t  off_zoff;     /*  40 */
  int64_t  off_sub_zoff; /*  48 */
  int64_t  off_data;     /*  56; the container's size is zoff[nblocks]                     */
} numarck_zindex_header;

/* Bytes a container can need for the blob whose header (host copy) is given; 0 if invalid. */
size_t numarck_zindex_bound(const void* blob_header_host);
/* Device workspace bytes numarck_deflate_index needs (81 per sub-block and about 3 KB per index
 * block); 0 if invalid. */
size_t numarck_zindex_workspace_bytes(const void* blob_header_host);
/* Deflates the index section of a compressed blob (device, with its header's host copy) into
 * zindex (device, zcap >= numarck_zindex_bound, 256-byte aligned). Asynchronous on stream;
 * the container's size is zoff[nblocks] (the 8 bytes at off_zoff + 8 * nblocks). */
int numarck_deflate_index(const void* blob, const void* blob_header_host, void* zindex,
                          size_t zcap, void* ws, size_t ws_bytes, numarck_stream_t stream);
/* Inflates the sub-blocks that cover elements [start, start + count) from a container (device,
 * zbytes long) into the index section of `blob` (device, laid out as blob_header_host says;
 * the other sections are not touched). Malformed data sets *status_dev (if non-NULL) to
 * NUMARCK_ERR_CORRUPT. Asynchronous on stream. */
int numarck_inflate_index(const void* zindex, size_t zbytes, const void* blob_header_host,
                          void* blob, int64_t start, int64_t count, int32_t* status_dev,
                          numarck_stream_t stream);

/* ---- served form: a request loop over resident time series (§I in-situ use, §IV.D) ----
 *
 * A server takes one caller-owned device buffer (the arena) and serves compress and
 * decompress requests for up to max_series time series from any number of client threads.
 * For each series it keeps in the arena the last reconstruction (the prev of the series' next
 * compression), the reconstruction the latest blob was compressed against, and the latest blob
 * (capacity for any B). The first compress request of a series only stores its timestep as the
 * reference (the caller keeps that timestep itself; completion.reference = 1); every later one
 * compresses the new timestep against the series' last reconstruction (Eq. 1 against R_{i-1}),
 * decodes the blob into the new reconstruction (Eq. 4) and copies the blob's used bytes to the
 * caller. A decompress request decodes all or part ([start, start + count)) of the series'
 * latest timestep from its latest blob into pinned host memory.
 *
 * Scheduling: the requests of one series run one at a time, in submission order. Across
 * series, the oldest request that can run starts as soon as one of `slots` CUDA streams is free
 * and its transient device buffers (a compression: the timestep and a workspace; a
 * decompression: its output; a series' first compression: the series' resident buffers) fit
 * in the arena's free space (first-fit); a younger request passes an older one that does not
 * fit only if the older one still fits afterwards. A request that cannot fit even with nothing
 * running completes with NUMARCK_ERR_CAPACITY. Results do not depend on what else runs: every
 * request has its own workspace and stream, and the kernels are deterministic.
 *
 * All host buffers (host_in, host_out) must be pinned (cudaHostAlloc / registered) and stay
 * valid until the request's completion is polled. Timestamps are seconds on the server's
 * steady clock. With dry_run = 1 no CUDA call is made and arena may be NULL: each request stage
 * takes dry_run_us microseconds (for tests of the scheduling on hosts without a GPU). */
typedef struct numarck_server numarck_server;

typedef struct numarck_server_config {
  void*   arena;          /* device buffer, 256-byte aligned, owned by the caller             */
  size_t  arena_bytes;
  int32_t slots;          /* requests in flight at once (one CUDA stream each), 1..64        */
  int32_t max_series;     /* series ids 0..max_series-1, 1..2^20                             */
  int32_t dry_run;        /* 0, or 1: no CUDA calls (see above)                              */
  int32_t dry_run_us;     /* dry run: duration of each request stage in microseconds         */
} numarck_server_config;

#define NUMARCK_REQ_COMPRESS   0
#define NUMARCK_REQ_DECOMPRESS 1

typedef struct numarck_request {
  int32_t kind;           /* NUMARCK_REQ_COMPRESS or NUMARCK_REQ_DECOMPRESS                   */
  int32_t series;         /* 0..max_series-1                                                  */
  numarck_params params;  /* compress: dtype, B (1..16), E, anchor, block size; decompress:    *
                           * dtype (must be the series')                                      */
  int64_t n;              /* elements of the series (fixed by its first timestep)            */
  const void* host_in;    /* compress: the new timestep, n elements of T, pinned             */
  void*   host_out;       /* compress: the blob; decompress: count elements of T; pinned     */
  size_t  host_out_cap;   /* bytes at host_out                                               */
  int64_t start, count;   /* decompress: elements [start, start + count) of the timestep     */
} numarck_request;

typedef struct numarck_completion {
  uint64_t id;            /* as returned by numarck_server_submit                             */
  int32_t status;         /* NUMARCK_OK or an error code (CAPACITY: host_out too small, or the *
                           * request can never fit in the arena; INVALID_ARG: n or dtype not   *
                           * the series', or a decompression before any compression)          */
  int32_t kind, series;
  int32_t reference;      /* 1: the series' first timestep, stored as its reference           */
  int32_t pad;
  uint64_t out_bytes;     /* bytes written to host_out                                        */
  double  t_submit, t_start, t_end;
} numarck_completion;

typedef struct numarck_server_stats {
  uint64_t submitted, started, completed;
  uint64_t deferred_memory;   /* admission attempts deferred for lack of arena space         */
  uint64_t arena_bytes, arena_used, arena_peak;
  int32_t  max_inflight, pad;
  double   now;
} numarck_server_stats;

/* Creates a server (starts its worker thread on the current device). Returns NULL and sets
 * *status (if non-NULL) on invalid configuration or CUDA errors. */
numarck_server* numarck_server_create(const numarck_server_config* cfg, int* status);
/* Queues a request (thread-safe, never blocks on the GPU); *id receives its id. Returns
 * NUMARCK_ERR_INVALID_ARG for malformed requests (series out of range, bad params, B = 0). */
int numarck_server_submit(numarck_server* s, const numarck_request* r, uint64_t* id);
/* Moves up to max completions (oldest first) to out, waiting up to wait_ms for the first one;
 * *got receives their number. */
int numarck_server_poll(numarck_server* s, numarck_completion* out, int max, int* got,
                        int wait_ms);
int numarck_server_get_stats(numarck_server* s, numarck_server_stats* out);
/* Runs every submitted request to completion, then frees the server's streams and events
 * (the arena stays the caller's). */
int numarck_server_destroy(numarck_server* s);

#ifdef __cplusplus
}  /* extern "C" */
#endif

#endif /* NUMARCK_H */
