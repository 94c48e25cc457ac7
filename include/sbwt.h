/*
 * sbwt.h -- C ABI of the GB300 set-bwte library (libsbwt.so).
 *
 * The library builds and incrementally extends the Burrows-Wheeler transform
 * of a set of strings (DNA reads) on one GPU, following set-bwte
 * (Pantaleoni, arXiv 1410.0562):
 *
 *   - The BWT of a string set S_0..S_{m-1} is the BWT of
 *     T = S_0 $_0 ... S_{m-1} $_{m-1} with $_0 < ... < $_{m-1} < c_1
 *     (Section 2, Eq. 1): B[i] = T[(SA[i]-1) mod n].  Terminators are
 *     ordered by global read index, which is the order reads were appended.
 *   - rank(c,k,B) = |{i<k : B[i]=c}| (Section 2, Eq. 2).
 *   - Each sbwt_append splits its reads into blocks of at most M suffixes
 *     (a read longer than M forms its own block) and adds each block in turn
 *     (Algorithm 1): ConstructSA of the block, B_int, ComputeRanks against
 *     the current index (Lemma 1 and Algorithm 2 of Section 4), the g[SA_int]
 *     reordering and Insert (Section 5).  All of these run as CUDA kernels;
 *     there is no CPU fallback.
 *
 * Conventions shared by every call:
 *   - Return value: SBWT_OK (0) or a negative SBWT_E* code; sbwt_strerror
 *     turns it into text.  On any error the index is left exactly as it was
 *     before the call.
 *   - A handle is not thread-safe: one call at a time per handle.
 *   - Host pointers are owned by the caller and only read (or written) during
 *     the call.  Device pointers must be device memory of the index's GPU.
 *   - Alphabet: 1 to 16 distinct bytes in strictly increasing byte order
 *     (c_1 < ... < c_sigma, Section 2), none of them '$' or 0.  Up to 4
 *     symbols are held as 2-bit codes (text and rank dictionary, half a byte
 *     per row of B); 5 to 16 symbols as 4-bit codes (one byte per row).
 *     sbwt_bwt_noalloc takes 1 to 4 symbols only.
 *   - Read set: `reads` holds the concatenated bytes of m reads and `offsets`
 *     m+1 non-decreasing uint64 values with offsets[0] = 0; read j is
 *     reads[offsets[j] .. offsets[j+1]).  Empty reads are allowed.
 *   - B is returned one byte per row: the alphabet byte, or '$' (0x24) for
 *     every terminator (all $_k share one output byte).
 */
#ifndef SBWT_H
#define SBWT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define SBWT_OK 0
#define SBWT_EINVAL (-1)   /* bad argument, byte outside the alphabet, bad offsets */
#define SBWT_ENOMEM (-2)   /* the HBM budget (or the device) cannot hold the result */
#define SBWT_ERANGE (-3)   /* output buffer too small; the needed size is reported */
#define SBWT_EDEVICE (-4)  /* a CUDA error, or a device-side wait that gave up */
#define SBWT_ENOTSUP (-5)  /* option the library does not support */
#define SBWT_EBUSY (-6)    /* the index is serving: only submit/wait are allowed */
#define SBWT_ETIMEDOUT (-7) /* sbwt_wait: the request is not done yet */
#define SBWT_EIO (-8)       /* sbwt_save / sbwt_load: the file cannot be written or read */

typedef struct sbwt_index sbwt_index; /* opaque, owned by the library */

/* Options for sbwt_create_ex.  Zero-initialise and set what you need. */
typedef struct {
    uint32_t index_bits;     /* width of the g / g_sa row indices: 32 or 64; 0 =
                                32 while the index stays below 2^32 - 1 rows, 64
                                beyond.  With 32, an append that would reach
                                2^32 - 1 rows returns SBWT_EINVAL. */
    uint64_t block_suffixes; /* M of Algorithm 1 (suffixes per block), at most
                                2^31; 0 = 2^24 */
    void *stream;            /* cudaStream_t every kernel is launched on; NULL =
                                a stream the library creates and owns */
    int32_t device;          /* CUDA device ordinal; -1 = the current device */
    uint32_t host_tier;      /* 0 or 1 = allowed, 2 = forbidden, 3 = always (the
                                dictionary lives in host memory from the first
                                append on, whatever the budget): when the HBM budget
                                cannot hold the rank dictionaries (B_ext and its
                                counters), the index keeps ONE dictionary, in mapped
                                pinned host memory, which the same kernels reach over
                                the host link (Section 5 keeps B_ext in system
                                memory) and Insert rewrites in place, from its top
                                down in chunks staged in HBM: about 4 bits per row of
                                B in host memory (3.25 with occ_sampling 256), and
                                only the per-block working set in HBM.  A byte
                                outside the alphabet is still refused with the index
                                unchanged; a device error during such an append
                                leaves the index unusable (SBWT_EDEVICE) until
                                sbwt_reset. */
    uint32_t occ_sampling;   /* rows per occurrence block of the rank dictionary
                                (Section 5 keeps counters every 128 symbols): 64,
                                128 or 256; 0 = 64.  64 is one 32-byte sector per
                                block (4 bits per row of B, one sector per rank
                                query); 128 and 256 hold 3.5 and 3.25 bits per row
                                and read two to four sectors per query.
                                Alphabets of 5 to 16 symbols take 64 only
                                (SBWT_ENOTSUP otherwise). */
    uint32_t reserved[6];    /* must be zero */
} sbwt_options;

/* Creates an empty index over `alphabet` (a NUL-terminated string of 1..16
 * bytes in strictly increasing order, see the conventions).  hbm_budget_bytes caps the device
 * memory the index may hold, its working buffers included (0 = no cap beyond
 * the device's free memory).  Device state is created lazily by the first
 * call that needs the GPU, so this call does not touch the GPU.
 * Errors: SBWT_EINVAL (bad alphabet, NULL out), SBWT_ENOMEM (host). */
int sbwt_create(const char *alphabet, size_t hbm_budget_bytes, sbwt_index **out);

/* sbwt_create with options; opt may be NULL (all defaults).
 * Errors: as sbwt_create, plus SBWT_EINVAL for an invalid option. */
int sbwt_create_ex(const char *alphabet, size_t hbm_budget_bytes, const sbwt_options *opt,
                   sbwt_index **out);

/* Appends m reads from HOST memory (Algorithm 1 over the new reads; Section 2
 * notes that new strings can be added at any time because suffixes never
 * cross a read).  The reads get the global ids n_reads .. n_reads+m-1, in
 * order.  Inputs are validated before the index changes: a byte outside the
 * alphabet or bad offsets give SBWT_EINVAL and leave the index unchanged.
 * Blocks until the index holds the new reads. */
int sbwt_append(sbwt_index *idx, const uint8_t *reads, const uint64_t *offsets, uint64_t m);
/* Like sbwt_append, but the m reads go BEFORE every read already in the
 * index: they take ids 0 .. m-1 (in the given order) and the old reads'
 * ids move up by m.  Section 2 notes that the order of insertion can be
 * reversed; this is that order: Algorithm 1 runs over the new blocks from
 * the last to the first, and Algorithm 2 starts every new read at i := 0, since a new
 * terminator is smaller than every old one.  The result equals one append
 * of (new reads ++ old reads).  Same arguments, conventions and errors as
 * sbwt_append. */
int sbwt_prepend(sbwt_index *idx, const uint8_t *reads, const uint64_t *offsets, uint64_t m);

/* As sbwt_append, but `d_reads` (offsets[m] bytes) and `d_offsets` (m+1
 * values) are DEVICE pointers on the index's GPU.  The offsets are checked
 * and the blocks planned on the device; only the block table comes back to
 * the host (the offsets themselves only for an append of more blocks than
 * that table holds).  Blocks until done. */
int sbwt_append_device(sbwt_index *idx, const uint8_t *d_reads, const uint64_t *d_offsets, uint64_t m);

/* Writes B (n bytes, see conventions) into host buffer `out` of `cap` bytes
 * and sets *n_out = n.  If cap < n returns SBWT_ERANGE with *n_out = n and
 * nothing written; out may be NULL when cap is 0. */
int sbwt_get_bwt(sbwt_index *idx, uint8_t *out, uint64_t cap, uint64_t *n_out);

/* rank(c, k, B) (Eq. 2) for c an alphabet byte or '$', 0 <= k <= n.
 * Errors: SBWT_EINVAL for another c or k > n. */
int sbwt_rank(sbwt_index *idx, uint8_t c, uint64_t k, uint64_t *out);

/* q rank queries at once: out[i] = rank(cs[i], ks[i], B); host arrays.
 * Errors: SBWT_EINVAL if any query is invalid (nothing written). */
int sbwt_rank_batch(sbwt_index *idx, const uint8_t *cs, const uint64_t *ks, uint64_t q, uint64_t *out);

/* FM-index counting: counts[i] = occurrences of pattern i in the reads
 * (overlapping ones included), by backward search over B (Lemma 1 applied to
 * the pattern: the rows of the suffixes that start with P[k..], from [0, n),
 * one LF step per symbol).  Pattern i is patterns[offsets[i] .. offsets[i+1])
 * in host memory; offsets has q+1 non-decreasing entries starting at 0.  A
 * pattern with a byte outside the alphabet occurs 0 times; the empty pattern
 * counts every suffix (n).  Errors: SBWT_EINVAL for bad offsets. */
int sbwt_count(sbwt_index *idx, const uint8_t *patterns, const uint64_t *offsets, uint64_t q, uint64_t *counts);

/* Number of rows n (symbols, terminators included) and reads m. */
int sbwt_size(const sbwt_index *idx, uint64_t *n, uint64_t *m);

/* Memory the index holds: in HBM (counted against the budget) and in the
 * pinned host tier. */
int sbwt_memory(const sbwt_index *idx, uint64_t *hbm_bytes, uint64_t *host_bytes);

/* Empties the index (n = m = 0) and keeps its device buffers for reuse. */
int sbwt_reset(sbwt_index *idx);

/* Frees everything the index holds.  NULL is a no-op. */
void sbwt_destroy(sbwt_index *idx);

/* Static text for a status code. */
const char *sbwt_strerror(int code);

/* The cudaStream_t the index launches on (creating device state if needed). */
int sbwt_get_stream(sbwt_index *idx, void **stream);

/* ---- intermediates of the last block (for checking each step) ----------
 * With capture on, every append keeps the arrays of its LAST block:
 *   SBWT_STAGE_SA   : SA_int, block-local text positions (uint32 each);
 *                     position of read j's symbol k is
 *                     sum_{l<j}(|P_l|+1) + k over the block's reads, its
 *                     terminator at k = |P_j| (Algorithm 1, ConstructSA)
 *   SBWT_STAGE_BINT : B_int, one byte per suffix in SA order: 0..sigma-1
 *                     for c_1..c_sigma, 255 for a terminator
 *   SBWT_STAGE_G    : g, per block text position, number of rows of the
 *                     index before the block that are smaller (Algorithm 2),
 *                     uint64 each
 *   SBWT_STAGE_GSA  : g_sa = g[SA_int], uint64 each
 * sbwt_get_stage copies one of them to host memory `out` (cap bytes),
 * *count_out = number of elements; SBWT_ERANGE if it does not fit. */
#define SBWT_STAGE_SA 0
#define SBWT_STAGE_BINT 1
#define SBWT_STAGE_G 2
#define SBWT_STAGE_GSA 3
int sbwt_set_capture(sbwt_index *idx, int on);
int sbwt_get_stage(sbwt_index *idx, int stage, void *out, uint64_t cap, uint64_t *count_out);

/* ---- batched form: CUDA-graph replay --------------------------------------
 * With replay on, every append is captured into a CUDA graph and launched as
 * one unit: the whole block pipeline of Algorithm 1 (every block's
 * ConstructSA, ComputeRanks, B_int/g_sa and Insert, on both streams) is one
 * graph launch.  The library keeps one instantiated graph per pipeline shape
 * (the sequence of kernels an append launches, which follows from its block
 * count and longest read) and updates it in place with each append's sizes,
 * buffers and index state, so appends of different reads into a growing
 * index reuse it.  sbwt_get_kernel_stats counts the graph launches, updates
 * and instantiations as "host:graph_launch", "host:graph_update" and
 * "host:graph_instantiate".  Results are identical with replay on or off.
 * Up to 8 graphs are kept; sbwt_destroy and turning replay off drop them.
 * Off by default. */
int sbwt_set_graph_replay(sbwt_index *idx, int on);

/* Bandwidths the index's kernels work against, measured on its device and
 * stream: H2D and D2H copies of 256 MB between pinned host memory and HBM
 * (the host link the host tier uses), and random 32-byte sector reads by a
 * kernel from mapped pinned host memory and from 1 GB of HBM (the access of
 * ComputeRanks and rank queries to a dictionary that is not in L2), in GB/s.
 * Allocates 256 MB of pinned host memory and 1 GB of HBM for the
 * measurement and frees them (outside the HBM budget).  Errors:
 * SBWT_EINVAL, SBWT_ENOMEM, SBWT_EDEVICE, SBWT_EBUSY. */
typedef struct {
    double h2d_gbs, d2h_gbs;   /* copies over the host link */
    double host_random_gbs;    /* random 32-byte reads from mapped pinned host memory */
    double hbm_random_gbs;     /* random 32-byte reads from HBM */
} sbwt_bandwidth;
int sbwt_measure_bandwidth(sbwt_index *idx, sbwt_bandwidth *out);

/* Block overlap (on by default): the suffix sort of each block runs on a
 * second stream, ahead of the ranking, gather and Insert of the blocks before
 * it, which keep their order on the index's stream (the overlap of the
 * paper's pipeline, Section 7, Figure 1, with the GPU doing every stage).
 * Off: the plain per-block loop of Algorithm 1, every step of every block in
 * turn on the index's stream.  Results are identical.  Waits for the index's
 * stream; SBWT_EBUSY while serving. */
int sbwt_set_block_overlap(sbwt_index *idx, int on);

/* Autotunes M (suffixes per block, Algorithm 1) for reads like the given
 * ones: builds their BWT with each candidate M (three times; the fastest of
 * the last two counts), keeps the fastest M in the index and reports it in
 * *best_out; ms_out, if not NULL, gets each candidate's time in ms (-1 when
 * it did not fit the HBM budget).  d_reads/d_offsets are device arrays as in
 * sbwt_append_device.  candidates NULL = {2^22 .. 2^27}.  The index is
 * emptied (sbwt_reset) before returning.  Errors: SBWT_EINVAL (bad
 * arguments, a candidate 0 or above 2^31), SBWT_ENOMEM (no candidate fits),
 * or the error of a failing append. */
int sbwt_autotune_block_suffixes(sbwt_index *idx, const uint8_t *d_reads, const uint64_t *d_offsets, uint64_t m,
                                 const uint64_t *candidates, int ncand, uint64_t *best_out, double *ms_out);

/* Launch shapes of the kernels whose best shape depends on the reads:
 * insert_threads is the CTA size of the 2-bit Insert (256 or 512 threads
 * per output superblock; 0 = 512 while a quarter or more of the result's
 * rows are new, else 256); rank_segment is the number of positions one
 * ComputeRanks thread walks for reads longer than twice it (256, 512 or
 * 1024; 0 = 256; shorter reads take one thread each).  Results are
 * identical for every shape.  sbwt_set_tile_shapes sets them (SBWT_EINVAL
 * for another value or a nonzero reserved field), sbwt_get_tile_shapes
 * reads them. */
typedef struct {
    uint32_t insert_threads;
    uint32_t rank_segment;
    uint32_t reserved[2]; /* must be zero */
} sbwt_tile_shapes;
int sbwt_set_tile_shapes(sbwt_index *idx, const sbwt_tile_shapes *shapes);
int sbwt_get_tile_shapes(const sbwt_index *idx, sbwt_tile_shapes *out);

/* Autotunes the tile shapes with the index's current M and sampling: builds
 * the BWT of the given device reads three times with each candidate (the
 * fastest of the last two counts), keeps the fastest in the index and copies
 * it to *best_out (may be NULL); ms_out, if not NULL, gets each candidate's
 * time (-1: did not fit the HBM budget).  candidates NULL = five shapes:
 * insert_threads 0, 256 and 512 with rank_segment 256, and rank_segment 512
 * and 1024.  The index is emptied before and after.  Errors: SBWT_EINVAL,
 * SBWT_EBUSY, SBWT_ENOMEM (no candidate fits), or a failing append's. */
int sbwt_autotune_tile_shapes(sbwt_index *idx, const uint8_t *d_reads, const uint64_t *d_offsets, uint64_t m,
                              const sbwt_tile_shapes *candidates, int ncand, sbwt_tile_shapes *best_out,
                              double *ms_out);

/* Autotunes M and the occurrence sampling together (Algorithm 1's block
 * size; Section 5's counter spacing): every pair of a block size from
 * block_suffixes[0 .. n_block) and a sampling from samplings[0 .. n_sampling)
 * (64, 128 or 256 rows) builds the BWT of the given device reads three times
 * (the fastest of the last two counts).  The fastest pair is kept in the
 * index and reported in *best_block_out and *best_sampling_out (either may
 * be NULL); ms_out, if not NULL, gets n_sampling x n_block times in ms, row
 * by sampling (-1: did not fit the HBM budget).  block_suffixes NULL =
 * {2^22 .. 2^27}; samplings NULL = {64, 128, 256} (64 alone for 5 to 16
 * symbols).  The index is emptied before and after.  Errors: SBWT_EINVAL
 * (bad arguments or candidates), SBWT_ENOTSUP (a sampling other than 64 for
 * 5 to 16 symbols), SBWT_EBUSY, SBWT_ENOMEM (no pair fits), or the error of
 * a failing append. */
int sbwt_autotune(sbwt_index *idx, const uint8_t *d_reads, const uint64_t *d_offsets, uint64_t m,
                  const uint64_t *block_suffixes, int n_block, const uint32_t *samplings, int n_sampling,
                  uint64_t *best_block_out, uint32_t *best_sampling_out, double *ms_out);

/* ---- per-kernel timing ---------------------------------------------------
 * With profiling on, every kernel launch is bracketed by CUDA events on the
 * index's stream.  sbwt_get_kernel_stats fills up to `cap` records (one per
 * kernel name, accumulated since the last sbwt_reset_kernel_stats) and sets
 * *n_out to the number of distinct kernels.  `bytes` is the algorithmic HBM
 * traffic the launches were sized for (reads + writes of their inputs and
 * outputs, counted once).  Launch counts are kept even with profiling off. */
typedef struct {
    char name[48];
    uint64_t launches;
    double ms;      /* summed event time; 0 with profiling off */
    double bytes;   /* summed algorithmic bytes */
} sbwt_kernel_stat;
int sbwt_set_profiling(sbwt_index *idx, int on);
/* Profiling on, with events only around launches of the kernel named
 * `kernel` (one of the names sbwt_get_kernel_stats reports): the least
 * instrumentation that still times that kernel. */
int sbwt_set_profiling_only(sbwt_index *idx, const char *kernel);
int sbwt_get_kernel_stats(sbwt_index *idx, sbwt_kernel_stat *out, int cap, int *n_out);
int sbwt_reset_kernel_stats(sbwt_index *idx);

/* ---- served form: continuous batching of append requests ---------------
 * sbwt_serve_start attaches a server to the index: requests submitted with
 * sbwt_submit are appended in arrival order (their reads get consecutive
 * global ids in that order, as if appended one by one).  Requests waiting
 * when a batch starts are coalesced into that batch (one append, so one pass
 * of Insert over the index for all of them), up to max_batch_bases bases
 * (0 = no cap); the next batch's copy to the device overlaps the running
 * batch's kernels.  A request with a byte outside the alphabet fails alone
 * (SBWT_EINVAL from sbwt_wait).  While serving, the other calls that use the
 * index return SBWT_EBUSY; sbwt_serve_stop finishes every submitted request
 * and detaches the server (sbwt_destroy does too). */
int sbwt_serve_start(sbwt_index *idx, uint64_t max_batch_bases);
/* Copies the request (host arrays, as in sbwt_append) and queues it;
 * *ticket names it.  Thread-safe.  Errors: SBWT_EINVAL (not serving, bad
 * offsets), SBWT_EBUSY (stopping), SBWT_EDEVICE (serving ended on a device
 * error). */
int sbwt_submit(sbwt_index *idx, const uint8_t *reads, const uint64_t *offsets, uint64_t m, uint64_t *ticket);
/* Waits up to timeout_us (0 = do not wait) for a request; returns its
 * status (SBWT_ETIMEDOUT if not done yet, and the ticket stays valid), the
 * global id of its first read and its latency from submit to commit in ms.
 * A finished ticket can be waited for once.  Thread-safe. */
int sbwt_wait(sbwt_index *idx, uint64_t ticket, uint64_t timeout_us, uint64_t *first_read_id, double *latency_ms);
/* Finishes the submitted requests and stops serving; returns SBWT_EDEVICE if
 * a device error ended serving early, else SBWT_OK. */
int sbwt_serve_stop(sbwt_index *idx);

/* ---- Persistence ---------------------------------------------------------
 * The paper keeps B_ext in memory for the whole construction (Section 5);
 * persisting it is an addition.  sbwt_save writes the committed index --
 * the rank dictionary of B (occurrence blocks of 64 rows, 64-bit superblock
 * counters, C[] as Lemma 1 uses them), n, m, the alphabet and the index
 * width -- to the file `path` (created or truncated), with a header and a
 * 64-bit FNV-1a checksum of everything before it.  Little-endian, as laid
 * out on the device (the same on x86-64 and Arm).  Errors: SBWT_EINVAL (NULL
 * argument), SBWT_EBUSY (serving), SBWT_EDEVICE, SBWT_EIO.
 *
 * sbwt_load creates a new index from such a file, as sbwt_create_ex with the
 * file's alphabet would (`opt` as there; its index_bits, when 0, is the
 * file's), and places the dictionary under `hbm_budget_bytes` (in the host
 * tier if the budget asks for it).  The loaded index answers rank, count and
 * get_bwt like the saved one, and later appends continue its read ids.  The
 * file is checked (magic, version, sizes, checksum) before any device work:
 * SBWT_EIO (cannot open or read), SBWT_EINVAL (not an index file, or damaged;
 * bad options), SBWT_ENOMEM, SBWT_EDEVICE.  On error *out is NULL. */
int sbwt_save(sbwt_index *idx, const char *path);
int sbwt_load(const char *path, size_t hbm_budget_bytes, const sbwt_options *opt, sbwt_index **out);

/* ---- BWT of a small read set without allocating -------------------------
 * The paper has no counterpart to this call.  It is for callers that cannot
 * allocate device memory: a process whose device memory is handed out by
 * another framework's pool, a service that forbids allocation after start-up
 * to keep its footprint and latency fixed, or a plug-in whose host owns the
 * allocator.  Everything else in this library allocates its buffers with
 * cudaMalloc; this call does not (no cudaMalloc, cudaFree or allocating
 * library routine).
 *
 * It writes B (see conventions) of the m reads in host memory `reads` /
 * `offsets` into host buffer `out` of `cap` bytes, *n_out = n = offsets[m] +
 * m; the result is byte-for-byte what sbwt_create + sbwt_append +
 * sbwt_get_bwt give for the same reads.  `stream` is the cudaStream_t to run
 * on (NULL = the default stream); the call returns when the result is in
 * `out`.
 *
 * Its working memory is one file-scope device array sized for at most
 * SBWT_NOALLOC_MAX_SUFFIXES suffixes (reads plus one terminator each), about
 * 18 MB, which every GPU that loads the library holds until the process
 * exits.  Larger read sets return SBWT_EINVAL.  The first call on a device
 * looks up the array's device address (set-up, once per device); make that
 * first call before any stream capture.  All calls share the array and it
 * keeps the last call's contents; two calls whose GPU work overlapped would
 * race, so this function holds a process-wide lock until its stream has
 * finished.  Errors: SBWT_EINVAL (bad alphabet or offsets, an alphabet of
 * more than 4 symbols, a byte outside the alphabet, more than
 * SBWT_NOALLOC_MAX_SUFFIXES suffixes), SBWT_ERANGE
 * (cap < n), SBWT_EDEVICE. */
#define SBWT_NOALLOC_MAX_SUFFIXES (1u << 18)
int sbwt_bwt_noalloc(const char *alphabet, const uint8_t *reads, const uint64_t *offsets, uint64_t m,
                     uint8_t *out, uint64_t cap, uint64_t *n_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SBWT_H */
