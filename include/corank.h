/*
 * corank.h -- C ABI of the GB300 co-rank / stable-merge library (libcorank.so).
 *
 * Implements, on one NVIDIA GB300 (sm_103a), the method of Siebert & Traeff,
 * "Perfectly load-balanced, optimal, stable, parallel merge":
 *   - co_rank (Algorithm 1, Section 2; correctness by Lemma 1): for an output
 *     rank of the stable merge of ordered arrays A[m] and B[n], the unique
 *     prefix lengths of A and B that form that output prefix;
 *   - stable_merge driven by it (Algorithm 2, Section 3): the output is cut
 *     into equal tiles, each tile's input windows are found by co_rank, and
 *     every tile (and every thread inside it) merges exactly the same number
 *     of elements (Proposition 2).
 *
 * NAMING.  The paper calls the output rank i and the co-ranks j (into A) and
 * k (into B).  This ABI calls the output rank k and the co-ranks i (into A)
 * and j (into B):  paper (i; j, k)  ==  ABI (k; i, j).  Always i + j == k.
 *
 * ORDER AND STABILITY.  Keys are compared with the natural order of their type
 * (signed for CR_KEY_I32/I64, unsigned for CR_KEY_U32/U64).  CR_KEY_F32/F64
 * keys are IEEE-754 binary32/binary64 values ordered by the standard's
 * totalOrder predicate (-NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN, NaNs
 * by payload; every bit pattern is a valid key).  OR-ing CR_KEY_DESC into a key
 * type reverses the order (A and B descending, largest key first).
 * CR_KEY_PAIR_U32/I32 keys are 64-bit words holding a (major, minor) pair
 * of 32-bit keys -- the major key in the high 32 bits, i.e. a little-endian
 * struct { minor; major; } -- ordered lexicographically.  The paper
 * states the method for any total order (Section 2); these are instances of
 * it.  The merge is stable in every order: equal keys keep their order inside
 * A and inside B, and an A element precedes every equal B element (second
 * condition of Lemma 1 is strict).  A and B must be sorted in the chosen
 * order; this is not checked on the hot path.  Unsorted input gives an
 * unspecified result but never an out-of-bounds access or a hang.
 *
 * MEMORY.  Every pointer argument marked "device" is a device pointer owned by
 * the caller; the library allocates nothing.  Key, payload, tag, gradient and
 * permutation arrays may start at any address aligned to their element size
 * (so a window A + i0 of a larger array is passed as it is; CR_EALIGN for a
 * pointer that is not).  Library-format buffers -- workspaces and the source
 * flags of recorded merge passes -- must be 16-byte aligned.  Outputs must
 * not overlap inputs (CR_EALIAS).  Sizes are element counts (int64), at most
 * 2^59 per array (CR_EINVAL beyond).
 *
 * STREAMS AND ERRORS.  Every call is asynchronous and stream-ordered on
 * `stream` (a cudaStream_t; NULL = the legacy default stream).  Argument
 * errors are returned at once and nothing is launched.  A failed launch gives
 * CR_ECUDA; cr_last_error() then holds the CUDA message (per host thread).
 * Device-side conditions (a bounded wait that gave up, an inconsistent
 * segment table) are recorded in the workspace's status word and returned by
 * cr_workspace_status().
 *
 * THREADS.  All entry points are thread-safe; the device and its properties
 * are those current on the calling host thread.
 */
#ifndef CORANK_H
#define CORANK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CR_OK = 0,
    CR_EINVAL = 1,        /* bad size, rank, type, null pointer with nonzero size */
    CR_EALIAS = 2,        /* an output range overlaps an input range */
    CR_EALIGN = 3,        /* a pointer is not aligned as its argument requires */
    CR_ENOSPACE = 4,      /* workspace smaller than the *_workspace_size answer */
    CR_ECUDA = 5,         /* a CUDA runtime call failed; see cr_last_error() */
    CR_ETIMEOUT = 6,      /* (device) a bounded wait inside a kernel gave up */
    CR_EUNSUPPORTED = 7,  /* valid request this build does not implement */
    CR_EINTERNAL = 8,     /* (device) inconsistent tile or segment table */
    CR_EBADSEG = 9        /* (device) segment offsets not monotone / out of range */
} cr_status;

typedef enum {
    CR_KEY_I32 = 0,
    CR_KEY_U32 = 1,
    CR_KEY_I64 = 2,
    CR_KEY_U64 = 3,
    CR_KEY_F32 = 4,   /* float bits, IEEE-754 totalOrder (see ORDER below) */
    CR_KEY_F64 = 5,   /* double bits, IEEE-754 totalOrder */
    CR_KEY_PAIR_U32 = 6, /* (major, minor) uint32 pair in one 64-bit word, major in
                            the high 32 bits; lexicographic order */
    CR_KEY_PAIR_I32 = 7, /* the same with int32 halves */
    CR_KEY_DESC = 256 /* flag, OR-ed into any of the above: descending order */
} cr_key_type;

/* cudaStream_t, passed as a plain pointer so this header needs no CUDA header. */
typedef void* cr_stream;

/* Short name of a status code ("CR_OK", ...). Never NULL. */
const char* cr_status_string(int status);

/* Detail of the last error returned on this host thread ("" if none). */
const char* cr_last_error(void);

/* ABI version (major * 100 + minor). */
int cr_abi_version(void);

/* Elements per tile (TILE) the merge kernels use for this key type and
 * payload width under the current (balanced-class) tile shape: every tile of a merge carries
 * exactly TILE output elements except the last one (per segment, for batched
 * calls).  Returns 0 for an invalid combination. */
int64_t cr_tile_size(int key_type, int val_bytes);

/* Tile shapes.  A tile is merged by NT consumer threads, each merging ILP
 * interleaved runs of IPT elements (TILE = NT * IPT * ILP; Algorithm 2's equal
 * blocks, one per tile, and equal per-thread shares inside it,
 * Proposition 2).  Several shapes are compiled;
 * the one used is chosen per (key size, payload width) -- for example by the
 * autotuner -- and applies to every later call of that combination in the
 * process.  Workspace sizes depend on it: query them after choosing, and do
 * not change the shape between cr_merge_partition and the cr_merge_tiles*
 * calls that use its table (a table made for another TILE is refused on the
 * device: CR_EINTERNAL from cr_workspace_status).  Changing the shape while
 * calls of that combination are being issued on other host threads is a
 * race. */
int cr_tile_shape_count(void);
/* NT, IPT and ILP of shape `shape` (CR_EINVAL if out of range; each output
 * pointer may be NULL). */
cr_status cr_tile_shape_info(int shape, int* nt, int* ipt, int* ilp);
/* Select `shape` for this key type and payload width (0, 4, 8);
 * CR_EUNSUPPORTED if its shared-memory footprint does not fit. */
cr_status cr_set_tile_shape(int key_type, int val_bytes, int shape);
/* Current shape for this key type and payload width (-1 if invalid). */
int cr_get_tile_shape(int key_type, int val_bytes);

/* Shapes are chosen per key type, payload width and class.  Single merges
 * take one of three geometry classes: 2 "small" when m + n <= 2^23 (few
 * tiles per CTA slot), else 1 "skewed" when one input is more than 16 times
 * longer than the other (16 * min(m, n) < max(m, n)), else 0 "balanced".
 * Batched calls take class 3 "batched" and merge passes (plain and recorded)
 * class 4 "pass".  cr_set_tile_shape sets every class (except, for payload
 * widths 4 and 8, the pass class when the shape's TILE exceeds 4096: a
 * recorded pass keeps a tile's flags in one CTA of its backward); these set
 * and read one (cls = 0 .. 4; CR_EINVAL / -1 for another value;
 * CR_EUNSUPPORTED for a pass-class shape over 4096 elements with payloads). */
cr_status cr_set_tile_shape_for(int key_type, int val_bytes, int cls, int shape);
int cr_get_tile_shape_for(int key_type, int val_bytes, int cls);
/* TILE a single merge of m and n elements uses (0 for invalid arguments). */
int64_t cr_tile_size_for(int key_type, int val_bytes, int64_t m, int64_t n);
/* TILE of class cls (0 .. 4, as above; 0 for invalid arguments).  Batched
 * calls use cls 3, merge passes cls 4. */
int64_t cr_tile_size_class(int key_type, int val_bytes, int cls);

/* ------------------------------------------------------------------------
 * co_rank -- Algorithm 1 (Section 2), Lemma 1.
 * For output rank k of the stable merge of A[m] and B[n], 0 <= k <= m + n,
 * the unique (i, j), i + j == k, such that
 *     (i == 0 || j == n || A[i-1] <= B[j])  and  (j == 0 || i == m || B[j-1] < A[i]).
 * The first k outputs of the merge are exactly the merge of A[0:i), B[0:j).
 * k == m + n (used by Algorithm 2 for the last block end) gives (m, n).
 * ------------------------------------------------------------------------ */

/* One rank, result on the host: *i_out = i, *j_out = j.  A, B: device, m and
 * n keys.  k outside [0, m+n] -> CR_EINVAL.  Synchronous: the search runs as
 * one kernel on `stream`, the two results are copied back and `stream` is
 * synchronised before the call returns (so it cannot be captured into a CUDA
 * graph; use cr_co_rank_async there).  The kernel writes into a two-word
 * result slot in the library's device image (nothing is allocated); calls
 * on one device take turns on it. */
cr_status cr_co_rank(int key_type, const void* A, int64_t m, const void* B, int64_t n,
                     int64_t k, int64_t* i_out, int64_t* j_out, cr_stream stream);

/* One rank, result written to device memory on `stream` without waiting:
 * d_ij[0] = i, d_ij[1] = j (d_ij: device, 8-byte aligned).  Same arguments
 * and errors as cr_co_rank otherwise. */
cr_status cr_co_rank_async(int key_type, const void* A, int64_t m, const void* B, int64_t n,
                           int64_t k, int64_t* d_ij, cr_stream stream);

/* cnt ranks d_k[0..cnt) (device) -> d_i, d_j (device, cnt each).  A rank
 * outside [0, m+n] gives i = j = -1 for that entry. */
cr_status cr_co_rank_many(int key_type, const void* A, int64_t m, const void* B, int64_t n,
                          const int64_t* d_k, int64_t cnt, int64_t* d_i, int64_t* d_j,
                          cr_stream stream);

/* ------------------------------------------------------------------------
 * Block-distributed co-rank: Algorithm 1 (Section 2) when A and B are spread
 * over the processing elements of Algorithm 2 in contiguous blocks, as in the
 * distributed-memory remark of Section 3: every key a search compares is a
 * remote point read.  One iteration of cnt searches is split into the parts
 * a process group runs between its collectives:
 *   1. cr_dist_co_rank_probes: the positions each live search reads next;
 *   2. cr_dist_co_rank_answer: every rank answers the probes that fall in
 *      its own block (0 elsewhere), and the group sums the answers (one
 *      all-reduce), which delivers every key exactly once;
 *   3. cr_dist_co_rank_step: one iteration of Algorithm 1 on those keys.
 * After at most ceil(log2(min(m, n) + 1)) + 1 iterations every search has
 * finished (the corrected iteration bound of Proposition 1 plus the final
 * check); cr_dist_co_rank_result reads the co-ranks and counts unfinished
 * searches.  The arithmetic runs in these kernels; the caller only moves
 * the probe positions and answers between ranks.
 *
 * State (device, int64, 6 * cnt entries, column by column): rank k, co-rank
 * i (into A), co-rank j (into B), the low bounds of i and j, and a finished
 * flag.  Probe arrays (device, int64, 2 * cnt entries each): pa[2q] = i - 1,
 * pa[2q+1] = i, pb[2q] = j - 1, pb[2q+1] = j of search q, -1 where that key
 * is not needed.  Answers (device, int64, as many as probes): the key's bits
 * (4-byte keys zero-extended).  All arrays 8-byte aligned; m, n are the
 * global lengths of A and B; key order as everywhere else.  Asynchronous on
 * `stream`.  A rank outside [0, m + n] gives a finished search with
 * i = j = -1.
 * ------------------------------------------------------------------------ */
cr_status cr_dist_co_rank_init(int64_t m, int64_t n, const int64_t* d_ranks, int64_t cnt,
                               int64_t* d_state, cr_stream stream);

cr_status cr_dist_co_rank_probes(int64_t m, int64_t n, const int64_t* d_state, int64_t cnt,
                                 int64_t* d_probe_a, int64_t* d_probe_b, cr_stream stream);

/* d_vals[q] = bits of blk[d_idx[q] - lo] when lo <= d_idx[q] < hi, else 0.
 * blk (device): this rank's block of A or B, the elements [lo, hi) of that
 * array. */
cr_status cr_dist_co_rank_answer(int key_type, const void* blk, int64_t lo, int64_t hi,
                                 const int64_t* d_idx, int64_t cnt, int64_t* d_vals,
                                 cr_stream stream);

/* d_vals_a / d_vals_b: the summed answers to d_probe_a / d_probe_b. */
cr_status cr_dist_co_rank_step(int key_type, int64_t m, int64_t n, const int64_t* d_vals_a,
                               const int64_t* d_vals_b, int64_t* d_state, int64_t cnt,
                               cr_stream stream);

/* d_i[q], d_j[q] = the co-ranks of search q; *d_live (device, one uint64) =
 * the number of searches not yet finished. */
cr_status cr_dist_co_rank_result(const int64_t* d_state, int64_t cnt, int64_t* d_i,
                                 int64_t* d_j, uint64_t* d_live, cr_stream stream);

/* ------------------------------------------------------------------------
 * stable_merge -- Algorithm 2 (Section 3) with fixed-size output tiles.
 * C[0, m+n) = stable merge of A[0, m) and B[0, n).
 * ------------------------------------------------------------------------ */

/* Workspace bytes a single merge of m + n elements needs (tile table and
 * status word).  val_bytes: 0 (keys only), 4 or 8. */
cr_status cr_merge_workspace_size(int key_type, int val_bytes, int64_t m, int64_t n,
                                  size_t* bytes);

/* Keys only.  C_tag (device, nullable): if given, C_tag[x] = source position
 * of C[x]: i for A[i], m + j for B[j] (requires m + n <= 2^32).  ws: device
 * workspace of at least cr_merge_workspace_size bytes, 16-byte aligned. */
cr_status cr_stable_merge(int key_type, const void* A, int64_t m, const void* B, int64_t n,
                          void* C, uint32_t* C_tag, void* ws, size_t ws_bytes,
                          cr_stream stream);

/* Key-value merge: payloads of val_bytes (4 or 8) bytes follow their keys and
 * are copied bit for bit (no floating-point operation touches them).
 * Ak/Av: m keys/payloads, Bk/Bv: n, Ck/Cv: m + n.  C_tag as above. */
cr_status cr_stable_merge_kv(int key_type, int val_bytes,
                             const void* Ak, const void* Av, int64_t m,
                             const void* Bk, const void* Bv, int64_t n,
                             void* Ck, void* Cv, uint32_t* C_tag,
                             void* ws, size_t ws_bytes, cr_stream stream);

/* Backward of the key-value merge with respect to the payloads.  The merge is
 * a permutation, so gA[i] = gC[position of A[i] in C] and gB[j] likewise
 * (bit copies of val_bytes each).  The permutation is not stored: the tile
 * co-ranks are recomputed from the keys Ak, Bk.  gC: m + n, gA: m, gB: n. */
cr_status cr_stable_merge_kv_backward(int key_type, int val_bytes,
                                      const void* Ak, int64_t m, const void* Bk, int64_t n,
                                      const void* gC, void* gA, void* gB,
                                      void* ws, size_t ws_bytes, cr_stream stream);

/* The two steps of cr_stable_merge[_kv] as separate calls (the variant of
 * Section 3 in which the co-ranks of all block boundaries are computed first
 * and shared, so each is searched once per call instead of once per block
 * end): cr_merge_partition writes the tile table of a merge of A[m], B[n]
 * into ws; cr_merge_tiles / cr_merge_tiles_backward then merge (or route
 * gradients) tile by tile from that table.  The table depends only on the
 * keys, m, n, key_type and val_bytes, so one partition can serve a forward
 * and a backward call.  The caller must pass the same A, B, m, n, key_type
 * and val_bytes to both steps and keep ws untouched in between; the tile
 * kernels check every record against the array bounds (CR_EINTERNAL via
 * cr_workspace_status) but cannot detect a table made for other keys. */
cr_status cr_merge_partition(int key_type, int val_bytes, const void* A, int64_t m,
                             const void* B, int64_t n, void* ws, size_t ws_bytes,
                             cr_stream stream);

/* Same table as cr_merge_partition, computed the way each processing element
 * of Algorithm 2 (Section 3) does it without synchronisation: every tile
 * co-ranks both of its ends itself with Algorithm 1, sharing nothing with
 * its neighbours.  Offered to compare the paper's two forms; the shared form
 * above is faster on GB300. */
cr_status cr_merge_partition_alg2(int key_type, int val_bytes, const void* A, int64_t m,
                                  const void* B, int64_t n, void* ws, size_t ws_bytes,
                                  cr_stream stream);

cr_status cr_merge_tiles(int key_type, int val_bytes, const void* Ak, const void* Av, int64_t m,
                         const void* Bk, const void* Bv, int64_t n, void* Ck, void* Cv,
                         uint32_t* C_tag, void* ws, size_t ws_bytes, cr_stream stream);

cr_status cr_merge_tiles_backward(int key_type, int val_bytes, const void* Ak, int64_t m,
                                  const void* Bk, int64_t n, const void* gC, void* gA, void* gB,
                                  void* ws, size_t ws_bytes, cr_stream stream);

/* ------------------------------------------------------------------------
 * Batched (segmented) merge: nseg independent merges in one persistent launch.
 * Segment s merges Ak[a_off[s], a_off[s+1]) with Bk[b_off[s], b_off[s+1])
 * into Ck[a_off[s] + b_off[s], a_off[s+1] + b_off[s+1]).
 * d_a_off, d_b_off: device int64 tables of nseg + 1 entries, a_off[0] ==
 * b_off[0] == 0, non-decreasing, a_off[nseg] <= a_total, b_off[nseg] <=
 * b_total (checked on the device: CR_EBADSEG via cr_workspace_status, and the
 * call then writes nothing).  a_total / b_total: lengths of Ak / Bk.
 * val_bytes 0 means keys only (Av, Bv, Cv ignored).
 * ------------------------------------------------------------------------ */
cr_status cr_batched_workspace_size(int key_type, int val_bytes, int64_t nseg,
                                    int64_t a_total, int64_t b_total, size_t* bytes);

cr_status cr_batched_merge_kv(int key_type, int val_bytes, int64_t nseg,
                              const int64_t* d_a_off, const int64_t* d_b_off,
                              const void* Ak, const void* Av, int64_t a_total,
                              const void* Bk, const void* Bv, int64_t b_total,
                              void* Ck, void* Cv, void* ws, size_t ws_bytes,
                              cr_stream stream);

/* Backward of cr_batched_merge_kv with respect to the payloads (val_bytes 4
 * or 8): gA[a_off[s] + i] = gC[position of that element in segment s], ... */
cr_status cr_batched_merge_kv_backward(int key_type, int val_bytes, int64_t nseg,
                                       const int64_t* d_a_off, const int64_t* d_b_off,
                                       const void* Ak, int64_t a_total,
                                       const void* Bk, int64_t b_total,
                                       const void* gC, void* gA, void* gB,
                                       void* ws, size_t ws_bytes, cr_stream stream);

/* ------------------------------------------------------------------------
 * Merge pass: one pass of a bottom-up stable merge sort.  X[0, N) holds
 * sorted runs of `width` elements; pair q merges X[2q*width, (2q+1)*width)
 * with X[(2q+1)*width, (2q+2)*width) (both cut at N) into the same range of
 * Y.  val_bytes 0, 4 or 8 (Xv/Yv ignored for 0).
 * ------------------------------------------------------------------------ */
cr_status cr_merge_pass_workspace_size(int key_type, int val_bytes, int64_t N, int64_t width,
                                       size_t* bytes);

cr_status cr_merge_pass(int key_type, int val_bytes, const void* X, const void* Xv, int64_t N,
                        int64_t width, void* Y, void* Yv, void* ws, size_t ws_bytes,
                        cr_stream stream);

/* Backward of cr_merge_pass for the payloads: X are the pass's INPUT keys,
 * gY (N payload gradients) -> gX (N). */
cr_status cr_merge_pass_backward(int key_type, int val_bytes, const void* X, int64_t N,
                                 int64_t width, const void* gY, void* gX,
                                 void* ws, size_t ws_bytes, cr_stream stream);

/* Recorded merge pass: the same forward as cr_merge_pass (val_bytes 4 or 8),
 * which also leaves in ws the pass's tile table and in `flags` one bit per
 * output telling which run of its pair it came from.  The backward
 * (cr_merge_pass_backward_recorded) then routes gradients from those bits
 * and reads no keys: per element it moves gY in, gX out and one bit, instead
 * of re-merging the keys.  The paper has no counterpart; it describes only
 * the forward merge.
 *
 * Layout of `flags` (uint32 words, 16-byte aligned, flag_words words): tile
 * t of the pass owns words [t*TILE/32, (t+1)*TILE/32); bit x % 32 of word
 * t*TILE/32 + x/32 is set when the tile's output x came from the pair's
 * second run (TILE = cr_tile_size_class(key_type, val_bytes, 4): merge
 * passes use the pass-class shape, at most 4096 elements).
 * Sizes: cr_merge_pass_record_size gives the workspace bytes and flag words
 * for (key_type, val_bytes, N, width) under the current tile shape.
 *
 * The backward must get the N, width, key_type and val_bytes of the forward,
 * with ws and flags untouched since and the tile shape unchanged; a table
 * made for another tile size or tile count is refused on the device
 * (CR_EINTERNAL via cr_workspace_status).  flags must not overlap Y, Yv or
 * the inputs (CR_EALIAS); too few words: CR_ENOSPACE. */
cr_status cr_merge_pass_record_size(int key_type, int val_bytes, int64_t N, int64_t width,
                                    size_t* ws_bytes, size_t* flag_words);

cr_status cr_merge_pass_record(int key_type, int val_bytes, const void* X, const void* Xv,
                               int64_t N, int64_t width, void* Y, void* Yv, uint32_t* flags,
                               size_t flag_words, void* ws, size_t ws_bytes, cr_stream stream);

/* gY (N payload gradients of the recorded pass's output) -> gX (N). */
cr_status cr_merge_pass_backward_recorded(int key_type, int val_bytes, int64_t N, int64_t width,
                                          const uint32_t* flags, size_t flag_words,
                                          const void* gY, void* gX, void* ws, size_t ws_bytes,
                                          cr_stream stream);

/* ------------------------------------------------------------------------
 * Run formation for a stable merge sort from unsorted input: every run of
 * cr_sort_run_length() (4096) consecutive elements of X[0, N) (the last one
 * may be shorter) is stably sorted into Y (payloads follow their keys, equal
 * keys keep their input order), so that cr_merge_pass can take over with
 * width cr_sort_run_length().  Same result as cr_merge_runs_block with width
 * 1.  The paper has no counterpart; it assumes sorted inputs.  The backward
 * routes gY to gX through the same in-run permutation, recomputed by sorting
 * the input keys X again.  Y must not overlap X; val_bytes 0, 4 or 8 (4 or 8
 * for the backward).
 * ------------------------------------------------------------------------ */
int64_t cr_sort_run_length(void);

cr_status cr_sort_runs(int key_type, int val_bytes, const void* X, const void* Xv, int64_t N,
                       void* Y, void* Yv, cr_stream stream);

cr_status cr_sort_runs_backward(int key_type, int val_bytes, const void* X, int64_t N,
                                const void* gY, void* gX, cr_stream stream);

/* Recorded run formation: the same forward as cr_sort_runs (val_bytes 4 or
 * 8) that also writes each run's permutation, perm[base + x] = index inside
 * the run of the input element that became output x (uint16, N entries,
 * 2-byte aligned, must not overlap the other arrays).  Its backward
 * cr_sort_runs_backward_recorded reads no keys: gX[base + perm[base + x]] =
 * gY[base + x] within every run.  It must get the perm written by the
 * forward for the same N (entries pointing outside their run are skipped). */
cr_status cr_sort_runs_record(int key_type, int val_bytes, const void* X, const void* Xv,
                              int64_t N, void* Y, void* Yv, uint16_t* perm, cr_stream stream);

cr_status cr_sort_runs_backward_recorded(int val_bytes, int64_t N, const uint16_t* perm,
                                         const void* gY, void* gX, cr_stream stream);

/* ------------------------------------------------------------------------
 * Allocation-free stable merge (the paper has no counterpart: this is a
 * deployment convenience of this library).
 * Same result as cr_stable_merge (keys only, optional C_tag), but it takes no
 * workspace: the tile table lives in a fixed 4 MiB array inside the library's
 * device image, which every GPU that loads the library holds until exit.
 * For callers that cannot call cudaMalloc or take memory from an allocator --
 * code running inside a host framework that owns every allocation, a
 * real-time loop that must not enter the allocator, a plug-in handed only its
 * input and output buffers.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current); make that first call
 *     before any stream capture begins.  Only a successful lookup is kept
 *     (a failed one is retried by the next call).  The address belongs to
 *     the device context it was found in: do not call this entry point
 *     again after cudaDeviceReset in the same process.
 *   - Size limit: m + n at most 131064 tiles of cr_tile_size_for(key_type,
 *     0, m, n) elements each (with the compiled-in shapes: 503,285,760
 *     elements for 4-byte keys, 234,866,688 for 8-byte keys; more with
 *     larger tiles selected).  Larger requests (including sizes whose sum
 *     would overflow) return CR_EINVAL and launch nothing.
 *   - A, B, C and C_tag need only be aligned to their element size.
 *   - Every call shares the array; calls whose kernels overlap on the GPU
 *     (other streams, other host threads) race and may give wrong output, so
 *     serialise them on one stream.  Device-side status is not reported for
 *     this entry point (cr_workspace_status needs a workspace).
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 * ------------------------------------------------------------------------ */
cr_status cr_stable_merge_noalloc(int key_type, const void* A, int64_t m, const void* B,
                                  int64_t n, void* C, uint32_t* C_tag, cr_stream stream);

/* ------------------------------------------------------------------------
 * Device-side status of the last call that used workspace `ws` on `stream`.
 * Synchronises `stream`, reads the status word and returns CR_OK,
 * CR_ETIMEOUT, CR_EINTERNAL or CR_EBADSEG (or CR_ECUDA if the read failed).
 * ------------------------------------------------------------------------ */
cr_status cr_workspace_status(const void* ws, cr_stream stream);

/* ------------------------------------------------------------------------
 * Merge block: the first passes of a merge sort done inside shared memory
 * (the paper has no counterpart; same result as those cr_merge_pass calls).
 * X[0, N) holds sorted runs of `width` (a power of two, 1 <= width <=
 * cr_merge_runs_block_length() / 2); every chunk of
 * cr_merge_runs_block_length() elements (4096; the last chunk may be
 * shorter) is merged into one sorted run of Y, i.e. the passes width, 2 width,
 * ..., up to the chunk length, in one read and one write of the arrays.
 * With width 1 (runs of one element: any input) this is run formation: the
 * chunk is sorted stably (ties keep input order); widths below 8 start from
 * groups of 8 sorted in registers.
 * val_bytes 0, 4 or 8.  With perm (uint16, N entries, 4 or 8 byte payloads
 * only) the chunk permutation is written: perm[base + x] = index inside the
 * chunk of the input element that became output x; its backward
 * cr_merge_runs_block_backward_recorded routes gY to gX through it without
 * keys.  Arrays aligned to their element size (CR_EALIGN); outputs must not
 * overlap inputs (CR_EALIAS); CR_EINVAL for a bad width, key type or payload
 * width.
 * ------------------------------------------------------------------------ */
int64_t cr_merge_runs_block_length(void);

cr_status cr_merge_runs_block(int key_type, int val_bytes, const void* X, const void* Xv,
                              int64_t N, int64_t width, void* Y, void* Yv, uint16_t* perm,
                              cr_stream stream);

cr_status cr_merge_runs_block_backward_recorded(int val_bytes, int64_t N, const uint16_t* perm,
                                                const void* gY, void* gX, cr_stream stream);

/* ------------------------------------------------------------------------
 * Debug check of the precondition (the hot path does not validate it): is
 * A[0, m) sorted in key_type's order (including float and descending orders)?
 * d_first (device, one int64) receives -1 when it is, else the smallest p
 * with A[p] before A[p-1] in that order.  ws: device scratch of at least 16
 * bytes (16-byte aligned); A aligned to its key size.  Asynchronous on
 * `stream`.
 * CR_EINVAL / CR_EALIGN for bad arguments.
 * ------------------------------------------------------------------------ */
cr_status cr_check_sorted(int key_type, const void* A, int64_t m, int64_t* d_first, void* ws,
                          size_t ws_bytes, cr_stream stream);

/* ------------------------------------------------------------------------
 * Test hook (the paper has no counterpart).  Every mbarrier wait inside the
 * merge kernels gives up after a time limit, records CR_ETIMEOUT in the
 * workspace status word and lets the kernel return.  This call runs that
 * path on purpose: a one-thread kernel waits, with the same bounded wait and
 * `limit_ns` (1 .. 10^8 ns), on a barrier nothing arrives at, then writes the
 * status word of ws (ws_bytes >= 16, 16-byte aligned); cr_workspace_status
 * must then return CR_ETIMEOUT.  d_elapsed_ns (device, nullable) receives the
 * time the wait took.  CR_EINVAL for bad arguments.
 * ------------------------------------------------------------------------ */
cr_status cr_selftest_bounded_wait(void* ws, size_t ws_bytes, uint64_t limit_ns,
                                   uint64_t* d_elapsed_ns, cr_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* CORANK_H */
