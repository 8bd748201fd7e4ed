/*
 * grim.h - C ABI of the GB300 seed-location filter (GRIM-Filter: Kim et al.,
 * BMC Genomics 2018, arXiv 1711.01177).
 *
 * The reference genome is cut into overlapping bins; every bin gets a
 * 4^q-bit existence bitvector over all q-grams ("tokens").  For a read and
 * a candidate bin the filter counts the read's tokens present in the bin
 * (the accumulation sum) and passes the location when the sum reaches
 * T = (L - q + 1) - q*E for E tolerated edits.
 *
 * Conventions for every entry point:
 *  - pointers named "device" are CUDA device pointers (or managed memory)
 *    on the current device; "host" pointers are ordinary host memory;
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream); every call only enqueues work on that stream and returns; the
 *    caller synchronises before reading outputs or freeing inputs;
 *  - the library never frees or keeps caller memory; the bank is owned by
 *    the library from grim_build_bank until grim_bank_free;
 *  - working memory (scratch) comes from a stream-ordered memory pool per
 *    device that the library owns: freed blocks stay cached for later calls
 *    until grim_release_scratch hands them back to the device;
 *  - every call returns a status code (GRIM_OK = 0).  Host-side argument
 *    checks return GRIM_EINVAL / GRIM_ENOTSUP without enqueuing anything.
 *    Problems found in the DATA on the device (a base code > 3, a bin id
 *    >= n_bins, decreasing offsets, an over-long read) never fault: the
 *    affected outputs are written as "discard" (pass 0, sum 0) and a flag is
 *    raised in the bank's status word, read and cleared by grim_bank_status.
 *
 * Base codes: A=0, C=1, G=2, T=3.  Token value: the q bases read as a
 * base-4 number, first base most significant.
 */
#ifndef GRIM_H
#define GRIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define GRIM_OK 0
#define GRIM_EINVAL 1    /* bad argument, found on the host */
#define GRIM_EDATA 2     /* bad input data, found on the device */
#define GRIM_ENOMEM 3    /* device allocation failed */
#define GRIM_ECUDA 4     /* a CUDA runtime call failed (see grim_last_cuda_error) */
#define GRIM_EOVERFLOW 5 /* an output list exceeded the capacity given */
#define GRIM_ETIMEOUT 6  /* a bounded device-side wait ran out */
#define GRIM_ENOTSUP 7   /* parameters outside what the kernels implement */
#define GRIM_ESCRATCH 8  /* the request needs more than grim_scan_noalloc's fixed scratch */
#define GRIM_EIO 9       /* a bank file could not be written, or is not a valid bank file */

/* ---- device status flags (grim_bank_status) --------------------------- */
#define GRIM_FLAG_BAD_BASE 0x1u    /* a read holds a code > 3 */
#define GRIM_FLAG_BAD_BIN 0x2u     /* a candidate bin id >= n_bins */
#define GRIM_FLAG_BAD_OFFSETS 0x4u /* read or candidate offsets decrease */
#define GRIM_FLAG_LONG_READ 0x8u   /* a read longer than GRIM_MAX_READ_LEN */
#define GRIM_FLAG_OVERFLOW 0x10u   /* a pair list exceeded its capacity */
#define GRIM_FLAG_TIMEOUT 0x20u    /* a bounded device-side wait ran out */

#define GRIM_MAX_Q 6               /* token sizes 1..6 (the paper sweeps 4-6, Sec. 6.1) */
#define GRIM_MAX_SCAN_Q 5          /* token sizes of the full-scan form */
#define GRIM_MAX_READ_LEN 65535    /* so that every sum fits 16 bits */

typedef struct grim_bank grim_bank;

/* Synchronise the current device and return the library pool's cached
 * scratch memory on it to the device.  Safe to call at any time. */
int grim_release_scratch(void);

/*
 * Diagnostic of the bounded waits in the library's tensor-core pipeline (the
 * full scan's mbarrier waits, which on expiry raise GRIM_FLAG_TIMEOUT, drain
 * and return instead of hanging): one thread runs the same wait for limit_ns
 * (1 ms .. 2 s, else GRIM_EINVAL) on a barrier that nothing ever completes.
 * Returns GRIM_ETIMEOUT when the wait gave up as designed (GRIM_OK would
 * mean it did not); the device and the context stay usable.  Synchronises
 * `stream`.  The paper has no counterpart.
 */
int grim_wait_selfcheck(unsigned long long limit_ns, void* stream);

/* Text for a status code (static storage). */
const char* grim_strerror(int status);

/* cudaError_t of the most recent GRIM_ECUDA / GRIM_ENOMEM on this thread. */
int grim_last_cuda_error(void);

/*
 * Host-side fault injection, so that callers and tests can walk the
 * library's error paths (GRIM_ENOMEM, GRIM_ECUDA and the clean-up behind
 * them) without making the GPU fail.  The paper has no counterpart.
 *   kind GRIM_FAULT_ALLOC:  the nth device or page-locked host allocation
 *        the library makes from now on fails as if memory were exhausted:
 *        nothing is allocated and the call making it returns GRIM_ENOMEM
 *        (grim_last_cuda_error() = cudaErrorMemoryAllocation).
 *   kind GRIM_FAULT_LAUNCH: the nth kernel launch from now on is made with
 *        an empty grid, which the CUDA runtime rejects before anything runs
 *        on the device; the call returns GRIM_ECUDA
 *        (grim_last_cuda_error() = cudaErrorInvalidConfiguration).
 *   kind GRIM_FAULT_NONE:   disarm.
 * One fault is armed at a time (a new one replaces it); events on every
 * host thread count towards it; it fires once and disarms itself.  nth >= 1
 * (else GRIM_EINVAL).  The environment variable GRIM_FAULT=alloc:N or
 * launch:N arms the same fault when the library is first used.
 * grim_fault_pending returns the armed kind (GRIM_FAULT_NONE once it has
 * fired) and, in *left (nullable), how many more events until it fires.
 * Neither call touches the GPU.
 */
/*
 * Roofline denominators measured on the current device: the rates the
 * benchmark divides its achieved figures by.  The paper has no counterpart.
 *   GRIM_PEAK_L2_READ        work = bytes of a buffer that fits the L2 (a
 *                            multiple of 16, <= 64 MiB), read 40 times with
 *                            16-byte L2-only loads by every SM; *units =
 *                            bytes read.
 *   GRIM_PEAK_E4M3           one CTA per SM issues `work` dense tcgen05 MMAs
 *                            of 128 x 256 x 32 (kind::f8f6f4, e4m3), both
 *                            operands in shared memory; *units = flops.
 *   GRIM_PEAK_MXF4           the same for kind::mxf4 (e2m1, K = 64, unit
 *                            block scales).
 *   GRIM_PEAK_MXF4_TMEM_A, GRIM_PEAK_E4M3_TMEM_A   the same with A in tensor
 *                            memory (the full scan's arrangement).
 *   GRIM_PEAK_MXF4_TMEM_A_N128, GRIM_PEAK_E4M3_TMEM_A_N128   the same with
 *                            N = 128.
 *   GRIM_PEAK_INT8_MMA_SYNC  `work` trips of 8 legacy mma.sync m16n8k32 s8 per
 *                            warp, 32 warps per SM; *units = integer ops.
 * *ms = CUDA-event time of the timed launch on `stream`, after one warm-up
 * launch.  Synchronises `stream`; scratch from the library's pool.
 * GRIM_ETIMEOUT if an MMA pipeline wait ran out (bounded, 2 s).
 */
#define GRIM_PEAK_L2_READ 1
#define GRIM_PEAK_E4M3 2
#define GRIM_PEAK_MXF4 3
#define GRIM_PEAK_MXF4_TMEM_A 4
#define GRIM_PEAK_E4M3_TMEM_A 5
#define GRIM_PEAK_INT8_MMA_SYNC 6
#define GRIM_PEAK_MXF4_TMEM_A_N128 7 /* the full scan's MMA shape: 128 x 128 x 64, A in tensor memory */
#define GRIM_PEAK_E4M3_TMEM_A_N128 8
int grim_peak(int kind, int64_t work, double* units, float* ms, void* stream);

#define GRIM_FAULT_NONE 0
#define GRIM_FAULT_ALLOC 1
#define GRIM_FAULT_LAUNCH 2
int grim_fault_inject(int kind, int64_t nth);
int grim_fault_pending(int64_t* left);

/*
 * Build the bank: the existence bitvector of every bin (Sec. 3.1, Fig. 2;
 * generated once per reference).
 *   ref2bit  device, (len+3)/4 bytes: base k in bits 2*(k%4) of byte k/4.
 *   len      number of bases, >= 1.
 *   q        token size, 1..GRIM_MAX_Q.
 *   bin_len  bases per bin core, >= 1.  n_bins = ceil(len / bin_len) must
 *            fit 32 bits.
 *   overlap  bases each bin extends past its core (>= 0).  Bin b spans
 *            [b*bin_len, min(len, (b+1)*bin_len + overlap)); a token belongs
 *            to the bin when all its bases lie in the span.  Choose
 *            overlap >= the longest read (plus tolerated insertions) so a
 *            read starting in a core fits in that bin (Sec. 3.2).
 *   out      host, receives the bank handle.
 * Layout in HBM: bin-major rows of row_words 32-bit words (row_words =
 * max(4, 4^q/32), 16-byte aligned rows); bit t of bin b is bit (t & 31)
 * of word b*row_words + (t >> 5).  Allocates the bank with cudaMalloc and
 * enqueues the build on `stream`.
 */
int grim_build_bank(const uint8_t* ref2bit, int64_t len, int q, int bin_len, int overlap, void* stream,
                    grim_bank** out);

/*
 * Recompute every row of an existing bank from a reference of the bank's
 * length (Sec. 3.1): the build of grim_build_bank without its allocation -
 * for a reference edited in place, or to time the build kernel alone.
 * ref2bit as for grim_build_bank, (len + 3) / 4 bytes with len the bank's.
 * Enqueues on `stream`; allocates nothing.
 */
int grim_build_bank_into(grim_bank* bank, const uint8_t* ref2bit, void* stream);

/* Geometry and device address of a bank (any output pointer may be NULL):
 * the bin partition and bitvector layout that grim_build_bank made from
 * Sec. 3.1 / Fig. 2 (bins of bin_len bases plus overlap, one 4^q-bit
 * existence bitvector each).  The query itself has no counterpart in the
 * paper. */
int grim_bank_info(const grim_bank* bank, int64_t* len, int64_t* n_bins, int* q, int* bin_len, int* overlap,
                   int64_t* row_words, const uint32_t** bits);

/* Synchronise `stream`, then read and clear the bank's device status word.
 * *flags (nullable) receives the GRIM_FLAG_* bits raised since the last
 * call by any call that used this bank.  Returns GRIM_EDATA if a data flag
 * is set, GRIM_EOVERFLOW / GRIM_ETIMEOUT for those flags, else GRIM_OK.
 * The paper has no counterpart: its filter assumes valid input (Sec. 3.2
 * is silent on codes other than A, C, G, T), and this call is how the
 * device-side checks of this library report what they found. */
int grim_bank_status(grim_bank* bank, void* stream, uint32_t* flags);

/* Free the bank (synchronises the device first). NULL is a no-op.  The
 * paper has no counterpart (its bitvectors live in the memory for as long
 * as the reference is mapped against, Sec. 3.1 / 4.2). */
int grim_bank_free(grim_bank* bank);

/*
 * Bank files: the bank depends only on the reference and (q, bin_len,
 * overlap), so it is built once and kept (the paper stores it with the
 * reference, Sec. 3.1).  The file is a 64-byte header (magic "GRIMBNK1",
 * geometry, payload size, a 64-bit checksum of the payload) followed by the
 * rows in their device layout, in the host's byte order.
 * grim_bank_save synchronises `stream`, then copies the rows out through a
 * pinned staging buffer; GRIM_EIO if the file cannot be written.
 * grim_bank_load validates the header and the file size before any device
 * work, allocates a bank on the current device and fills it; GRIM_EIO for a
 * file that cannot be read, is not a bank file, has the wrong size or fails
 * its checksum (no bank is returned then).  Synchronises `stream`.
 */
int grim_bank_save(const grim_bank* bank, const char* path, void* stream);
int grim_bank_load(const char* path, void* stream, grim_bank** out);

/*
 * Gather-form filter: the Filter Bitmask Generator of Sec. 3.3 over a
 * candidate list (the seed locations a read mapper found), implementing the
 * five steps of Sec. 3.2 / Fig. 3 for every (read, candidate bin) pair.
 *   reads         device u8 codes 0..3, read r = reads[read_offsets[r] ..
 *                 read_offsets[r+1]); length <= GRIM_MAX_READ_LEN.
 *   read_offsets  device int64, n_reads + 1 entries, non-decreasing.
 *   n_reads       >= 0 (0 enqueues nothing).
 *   cand_bins     device u32 bin ids; read r's candidates are
 *                 cand_bins[cand_offsets[r] .. cand_offsets[r+1]).
 *   cand_offsets  device int64, n_reads + 1 entries, non-decreasing.
 *   E             device u16, tolerated edits per read.
 *   pass          device u8 output aligned with cand_bins: 1 = align this
 *                 location, 0 = discard (the seed location filter bitmask,
 *                 one byte per location).
 *   sums          device u16 output aligned with cand_bins, or NULL.
 * Duplicate candidates are checked independently; a read shorter than q
 * has sum 0 and passes iff its threshold is <= 0.  One launch, in which
 * each CTA works through the reads holding an equal share of the work; it
 * keeps no device state besides the bank's status word, so calls that
 * overlap on the GPU (other streams) are independent.
 */
int grim_filter(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
                const uint32_t* cand_bins, const int64_t* cand_offsets, const uint16_t* E, uint8_t* pass,
                uint16_t* sums, void* stream);

/*
 * grim_filter from HOST memory: every pointer below is host memory (reads,
 * read_offsets, cand_bins, cand_offsets, E in; pass out), with the meanings
 * of grim_filter.  The reads are processed in chunks of chunk_reads (<= 0:
 * an eighth of the reads, at least 65,536, the last eighth in four
 * quarters): each chunk's inputs are copied in and its pass bytes copied
 * out on two streams of the library's, while the filter runs on `stream`,
 * so that the copies of one chunk overlap the filtering of another.  The
 * two copy streams and their events are created by the first call on a
 * device and kept for later ones (a call made while another host thread
 * uses them creates its own).  Page-locked host buffers let the copies
 * overlap; pageable ones work but are copied synchronously.  Synchronises
 * `stream` (pass is complete on return).  Device memory: two chunk slots
 * from the library's pool.  A chunk whose end offset (read or candidate)
 * lies below its start offset gives GRIM_EINVAL before any copy; other
 * decreasing offsets are flagged on the device as for grim_filter.
 */
int grim_filter_host(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
                     const uint32_t* cand_bins, const int64_t* cand_offsets, const uint16_t* E, uint8_t* pass,
                     int64_t chunk_reads, void* stream);

/*
 * Launch shape of the batched filter.  Zero fields take defaults.
 */
typedef struct grim_tune {
    int32_t warps_per_cta;   /* 4 or 8 (default 8) */
    int32_t reads_per_claim; /* reads a warp claims from the work counter at a time (default 1) */
    int32_t ctas_per_sm;     /* resident CTAs per SM, up to the occupancy limit (default: the limit) */
    int32_t use_graph;       /* 1: capture the launches in a CUDA graph, replayed by identical calls */
    int64_t batch_reads;     /* reads per launch (default 262,144) */
} grim_tune;

/*
 * Batched gather filter: the five steps of Sec. 3.2 / Fig. 3 for every
 * (read, candidate bin) pair, as in grim_filter, with the same outputs,
 * computed by one
 * launch per batch of `batch_reads` reads in which every warp claims reads
 * from a device work counter, so reads of uneven length and uneven
 * candidate lists balance across the GPU.  With use_graph, the call's
 * launches are captured once into a CUDA graph and an identical later call
 * (same pointers, sizes, tune and stream) replays it; a stream that is
 * already capturing simply records the launches.  tune == NULL uses the
 * last grim_autotune result for this bank's q on this device, else the
 * defaults with use_graph = 1.  The graph cache is host state of the bank:
 * calls on one bank from several host threads must be serialised.  The
 * work counters live in the bank: batched calls on one bank that overlap
 * on the GPU without a graph of their own must be serialised.  The
 * batching, the work counter and the graph have no counterpart in the
 * paper, whose filter logic checks one read at a time (Sec. 4.2).
 */
int grim_filter_batched(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
                        const uint32_t* cand_bins, const int64_t* cand_offsets, const uint16_t* E, uint8_t* pass,
                        uint16_t* sums, const grim_tune* tune, void* stream);

/*
 * Autotuner of the batched filter: times every launch shape it knows
 * (warps per CTA x reads per claim x CTAs per SM) on the first batch of the
 * given workload, writes the fastest to *out (host), and remembers it for
 * grim_filter_batched(tune = NULL) with this bank's q on this device.
 * Synchronises `stream`; `pass` is overwritten.
 */
int grim_autotune(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
                  const uint32_t* cand_bins, const int64_t* cand_offsets, const uint16_t* E, uint8_t* pass,
                  grim_tune* out, void* stream);

/*
 * Per-batch choice between the two forms (candidate density).  The gather
 * form costs about one bank row per candidate; the full scan costs
 * n_reads x n_bins small contractions whatever the candidates, so it only
 * pays off when candidate lists cover a large share of the bins.
 * grim_choose_form writes GRIM_FORM_GATHER or GRIM_FORM_SCAN to *form
 * (host) for a batch of n_reads reads with n_checks candidates, from a cost
 * model that uses the gather rate last measured by grim_autotune for this
 * bank's q on this device (a default otherwise) and the full scan's
 * tensor-core rate.
 */
#define GRIM_FORM_GATHER 0
#define GRIM_FORM_SCAN 1
int grim_choose_form(const grim_bank* bank, int64_t n_reads, int64_t n_checks, int* form);

/*
 * Dispatching filter: grim_filter's pass bytes (no sums), computed batch by
 * batch (batch_reads reads, <= 0: 262,144) with the form grim_choose_form
 * picks.  A scanned batch's passing pairs are joined back onto its
 * candidates on the device, so both forms give the same bytes.  Gathered
 * batches use the launch shape grim_autotune chose for this bank's q on
 * this device (the defaults before it has run), without graphs; a run of
 * consecutive gathered batches is one launch.  Reads every batch's
 * candidate count from the device up front (synchronising `stream` once,
 * and once more per scanned batch) and takes the scan's working memory and
 * a small bounds array from the library's pool.
 * *n_scanned (host, nullable) receives the number of reads that went
 * through the full scan.
 */
int grim_filter_auto(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
                     const uint32_t* cand_bins, const int64_t* cand_offsets, const uint16_t* E, uint8_t* pass,
                     int64_t batch_reads, int64_t* n_scanned, void* stream);

/*
 * Full-scan form: the filter of Sec. 3.2 for every read against every bin
 * of the window [bin_begin, bin_end) (the paper's bin window, Sec. 6.1,
 * with every bin checked), computed as the contraction
 * Sum[r, b] = sum_t count_r(t) * bit_b(t) on the tcgen05 tensor cores
 * (exact: small-integer products and sums in f32).
 *   reads, read_offsets, n_reads, E   as for grim_filter.
 *   bin_begin, bin_end  0 <= bin_begin <= bin_end <= n_bins.
 *   pair_read, pair_bin device u32 outputs, capacity `cap` entries each;
 *                       passing pairs (Sum >= T) in no particular order.
 *   pair_sum            device u16 output (cap entries) or NULL.
 *   cap                 >= 0; pairs beyond cap are counted, not written,
 *                       and raise GRIM_FLAG_OVERFLOW.
 *   n_pairs             device int64, receives the number of passing pairs
 *                       (which may exceed cap).
 *   read_pass           device u32 [n_reads] or NULL: passing bins per read.
 * Token sizes 1..5 (GRIM_ENOTSUP above).  Allocates its scratch with
 * the library's pool, ordered on `stream`, and frees it the same way.
 */
int grim_scan(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
              const uint16_t* E, int64_t bin_begin, int64_t bin_end, uint32_t* pair_read, uint32_t* pair_bin,
              uint16_t* pair_sum, int64_t cap, int64_t* n_pairs, uint32_t* read_pass, void* stream);

/*
 * grim_scan_noalloc - grim_scan that allocates no device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they call the filter, for example a
 * process whose device memory is all owned by its own pool allocator (so an
 * allocation by this library could fail or compete with that pool), or
 * a service that fixes its device footprint at start-up and must not grow
 * it while serving.  Arguments, outputs and results are those of grim_scan.
 *
 * Its working memory is one array of GRIM_SCAN_NOALLOC_SCRATCH_BYTES
 * (64 MiB) compiled into the library: every GPU on which the library is
 * loaded holds it until the process exits.  A call needing more is
 * rejected with GRIM_ESCRATCH before anything is enqueued; the need is
 * 256 + sum over c = 0 .. 3 of ceil(n_reads / (256 >> c)) * 256 * K / 2
 * bytes (K = max(256, 4^q)) plus two small index arrays per c, which allows
 * at most 8,672 reads per call at q = 5 and 34,336 at q <= 4.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any
 * stream capture.  Every call uses the same array and finds the previous
 * call's contents in it (each call clears what must start at zero), so
 * calls whose work overlaps on the GPU - on different streams or from
 * different host threads - race on it: the caller must serialise them.
 */
/* The tcgen05 MMA kind the full scan runs on ("f8f6f4": e4m3 operands, or
 * "mxf4": e2m1 operands with unit block scales); static storage.  The paper
 * has no counterpart. */
const char* grim_scan_mma_kind(void);

#define GRIM_SCAN_NOALLOC_SCRATCH_BYTES (64ull << 20)
int grim_scan_noalloc(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
                      const uint16_t* E, int64_t bin_begin, int64_t bin_end, uint32_t* pair_read, uint32_t* pair_bin,
                      uint16_t* pair_sum, int64_t cap, int64_t* n_pairs, uint32_t* read_pass, void* stream);

/* ---- seed locations: the mapper's steps either side of the filter ------ */

/*
 * Seed location table of a reference (the hash table a seed-and-extend
 * mapper indexes with each seed, Sec. 1 / Fig. 1 step 3): the start
 * position of every k-mer, grouped by k-mer value in CSR form.
 *   ref2bit  device, 2-bit packed reference (base i in bits 2*(i%4) of
 *            byte i/4), as for grim_build_bank.
 *   len      bases, k <= len <= 2^32 - 1 (positions are u32).
 *   k        1..15 (keys index 4^k + 1 u32 offsets: 67 MB for k = 12).
 *   *out     receives the table (library-owned until grim_seed_index_free).
 * Device memory: 4 * (4^k + 1) + 4 * (len - k + 1) bytes, plus 4 * 4^k
 * bytes of stream-ordered scratch during the build.  The order of the
 * positions of one k-mer is not specified.  Enqueues on `stream`.
 */
typedef struct grim_seed_index grim_seed_index;
int grim_seed_index_build(const uint8_t* ref2bit, int64_t len, int k, void* stream, grim_seed_index** out);

/* Table metadata and zero-copy device views (offsets: 4^k + 1 u32,
 * positions: len - k + 1 u32).  Any output pointer may be NULL. */
int grim_seed_index_info(const grim_seed_index* idx, int64_t* len, int* k, const uint32_t** offsets,
                         const uint32_t** positions);

/* Free the table (synchronises the device first).  NULL is a no-op. */
int grim_seed_index_free(grim_seed_index* idx);

/*
 * Candidate bins of every read from its exact seed locations: what the
 * mapper sends to the filter with each read (Sec. 3.3: only the bins that
 * hold a potential seed location are checked).
 *   Seeds: the read's non-overlapping k-mers at offsets 0, k, 2k, ...
 *   (o + k <= L); a seed holding a code > 3 has no locations.  A location p
 *   of the seed at offset o puts the read's start at p - o and votes for
 *   the bin whose core holds max(0, p - o) (at most n_bins - 1).  The
 *   distinct voted bins are the read's candidates; when there are more
 *   than `cap`, the cap bins with the most votes are kept, equal votes
 *   going to the lower bin id.  Each read's list is ascending.
 *   reads, read_offsets, n_reads  as for grim_filter.
 *   bin_len, n_bins   the bank's geometry (n_bins < 2^32).
 *   cap               >= 1.
 *   cand_bins         device u32 output, `capacity` entries (may be NULL
 *                     when capacity is 0).
 *   cand_offsets      device int64 output, n_reads + 1 entries (CSR,
 *                     cand_offsets[0] = 0); always written in full.
 *   *n_cands          host: the total number of candidates.
 * Returns GRIM_EOVERFLOW when the total exceeds `capacity` (then only the
 * first `capacity` bins are written; call again with a larger buffer).
 * Unlike the filter entry points this call SYNCHRONISES `stream`: reads are
 * processed in batches whose vote scratch (12 bytes per seed location,
 * library's pool) is sized from per-read location counts read back to
 * the host.
 */
int grim_seed_candidates(const grim_seed_index* idx, const uint8_t* reads, const int64_t* read_offsets,
                         int64_t n_reads, int bin_len, int64_t n_bins, int cap, uint32_t* cand_bins,
                         int64_t capacity, int64_t* cand_offsets, int64_t* n_cands, void* stream);

/*
 * Seed Location Checker (Sec. 3.3, Fig. 4 steps 2-3): the locations whose
 * filter bit is 1, in candidate order, with the reference segment the
 * aligner receives for each - the bin's span [b * bin_len,
 * min(len, b * bin_len + bin_len + overlap)).
 *   bank              the bank the mask was computed with (geometry).
 *   cand_bins, cand_offsets, n_reads   the candidate lists (CSR,
 *                     cand_offsets[0] = 0, cand_offsets[n_reads] = n_cands).
 *   pass              device u8 [n_cands]: the filter bitmask.
 *   loc_read, loc_bin device u32 outputs, loc_begin, loc_end device int64
 *                     outputs (each of the two may be NULL: not written;
 *                     both are needed with segments), `capacity` entries.
 *   segments          device u8 [capacity * seg_stride] or NULL: row i holds
 *                     the base codes of location i's span, then code 4 up
 *                     to seg_stride (a span longer than seg_stride is cut);
 *                     needs ref2bit (device, 2-bit packed reference).
 *   *n_loc            device int64: the number of passing locations (which
 *                     may exceed capacity; outputs beyond it are not written).
 * A passing candidate whose bin id is >= n_bins gets the empty span [0, 0)
 * and raises GRIM_FLAG_BAD_BIN; cand_offsets[n_reads] != n_cands raises
 * GRIM_FLAG_BAD_OFFSETS.  Enqueues on `stream` (stream-ordered scratch).
 */
int grim_locate(const grim_bank* bank, const uint8_t* ref2bit, const uint32_t* cand_bins,
                const int64_t* cand_offsets, int64_t n_reads, int64_t n_cands, const uint8_t* pass,
                uint32_t* loc_read, uint32_t* loc_bin, int64_t* loc_begin, int64_t* loc_end, uint8_t* segments,
                int64_t seg_stride, int64_t capacity, int64_t* n_loc, void* stream);

/*
 * Edit budgets from an error rate (Sec. 3.4: the threshold tolerates E
 * edits, E the read length times the error rate; Sec. 6.1 uses a rate of
 * 0.05): E[r] = floor(num * L_r / den), or the ceiling when round_up != 0,
 * in exact integer arithmetic, with L_r = read_offsets[r+1] -
 * read_offsets[r] (a negative length gives 0, a length above
 * GRIM_MAX_READ_LEN counts as GRIM_MAX_READ_LEN + 1 — the filter rejects
 * such reads — and results above 65535 are saturated).
 * read_offsets: device i64 [n_reads + 1]; E: device u16
 * [n_reads], written.  num >= 0 and den >= 1, else GRIM_EINVAL.  Enqueues
 * on `stream`.
 */
int grim_fill_E_rate(const int64_t* read_offsets, int64_t n_reads, int32_t num, int32_t den, int32_t round_up,
                     uint16_t* E, void* stream);

/*
 * The seed location filter bitmask of Sec. 3.3 at one bit per location:
 * bit i % 32 of bits[i / 32] is 1 iff pass[i] != 0 (device u8 [n] in,
 * device u32 [ceil(n / 32)] out; the unused high bits of the last word are
 * 0).  Enqueues on `stream`.
 */
int grim_pack_mask(const uint8_t* pass, int64_t n, uint32_t* bits, void* stream);

/* ---- verification: the aligner's check and the paper's quality metrics -- */

/*
 * Edit distance of each location's read against its bin's span: the fewest
 * substitutions, insertions and deletions that turn the read into some
 * substring of the span [b * bin_len, min(len, b * bin_len + bin_len +
 * overlap)) (semi-global, Sellers' recurrence; computed with Myers'
 * bit-vector form).  A location results in a mapping (Sec. 5: locations
 * that "do not result in a mapping" after alignment count against the
 * filter) when the distance is <= the read's E.
 *   bank        geometry of the spans; ref2bit: device, the 2-bit packed
 *               reference the bank was built from.
 *   reads, read_offsets, n_reads   as for grim_filter (codes > 3 match
 *               nothing).
 *   loc_read, loc_bin   device u32 [n_loc]: the locations (for example the
 *               outputs of grim_locate).
 *   dist        device u16 output [n_loc] (distances above 65,534 read
 *               65,535).
 * Reads up to 512 bases; a longer read, a read id >= n_reads, a bin id >=
 * n_bins or decreasing offsets give 65,535 and raise the bank's
 * GRIM_FLAG_LONG_READ / BAD_OFFSETS / BAD_BIN flag.  Enqueues on `stream`.
 */
int grim_verify(const grim_bank* bank, const uint8_t* ref2bit, const uint8_t* reads, const int64_t* read_offsets,
                int64_t n_reads, const uint32_t* loc_read, const uint32_t* loc_bin, int64_t n_loc, uint16_t* dist,
                void* stream);

/*
 * Counts over n locations (device u64 counts[4], overwritten):
 *   counts[0] passing (pass byte != 0; every location when pass is NULL),
 *   counts[1] passing without a mapping (dist > E[read]),
 *   counts[2] rejected,
 *   counts[3] rejected with a mapping (dist <= E[read]).
 * The paper's "false negative rate" is counts[1] / counts[0]; its zero-miss
 * guarantee is counts[3] == 0 (no correct mapping filtered out); with one
 * location per candidate bin, counts[0] / (reads x n_bins) is the average
 * read existence of Sec. 6.1.
 *   pass       device u8 [n] or NULL; dist: device u16 [n] (grim_verify);
 *   loc_read   device u32 [n]; E: device u16 [n_reads].
 * Enqueues on `stream`.
 */
int grim_verify_stats(const uint8_t* pass, const uint16_t* dist, const uint32_t* loc_read, const uint16_t* E,
                      int64_t n_reads, int64_t n, unsigned long long* counts, void* stream);

/* ---- the mapper's path around the filter, overlapped --------------------- */

/*
 * Seed candidates -> filter -> Seed Location Checker -> edit distance of
 * every passing location, over batches of batch_reads reads (<= 0: 2^20),
 * with the aligner's work on one batch overlapping the filter's work on the
 * next (Sec. 4.2 / 6.1: alignment proceeds while the Filter Bitmask
 * Generator moves on, with a double-buffered bitmask between them).  The
 * filter steps run on `stream`, the distances on `align_stream` (NULL: a
 * stream created for the call at the device's lowest priority; a caller's
 * own align_stream is best given a lower priority than `stream`).
 *   bank, idx, ref2bit   the bank, the seed table (grim_seed_index_build)
 *                        and the 2-bit reference, of the same reference.
 *   reads, read_offsets, n_reads (< 2^32), E   as for grim_filter.
 *   cap                  the candidate cap of grim_seed_candidates.
 *   loc_read, loc_bin    device u32 outputs, loc_dist device u16 output,
 *                        `capacity` entries each: every passing location in
 *                        read order (candidate order within a read) with its
 *                        semi-global edit distance (grim_verify); a location
 *                        results in a mapping when loc_dist <= E[read].
 *   *n_loc               host: the number of passing locations.
 * Returns GRIM_EOVERFLOW when n_loc > capacity (the first `capacity` are
 * written).  Synchronises both streams; working memory (library pool): two
 * candidate slots sized to the largest batch (5 bytes per candidate each:
 * 1.25 x the most candidates per read seen by earlier grim_seed_candidates
 * calls with `idx`, at least 512 per read; a batch needing more grows its
 * slot and is redone), plus the scratch of the steps it calls.
 */
int grim_map(const grim_bank* bank, const grim_seed_index* idx, const uint8_t* ref2bit, const uint8_t* reads,
             const int64_t* read_offsets, int64_t n_reads, const uint16_t* E, int cap, int64_t batch_reads,
             uint32_t* loc_read, uint32_t* loc_bin, uint16_t* loc_dist, int64_t capacity, int64_t* n_loc,
             void* stream, void* align_stream);

#ifdef __cplusplus
}
#endif

#endif /* GRIM_H */
